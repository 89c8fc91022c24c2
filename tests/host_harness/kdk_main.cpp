// Host driver for the kick-drift-kick orbit body of k_orbit.cu (integration, mirrors, projection and the
// run-length binning into integer counts), compiled for the CPU so that the benchmark's per-orbit path can
// be compared with the oracle without a GPU.  Input file: 16 model scalars (as the adaptive integrator's
// driver; P[13] unused), 12 grid scalars, then n x 6 initial conditions (doubles).  Output: the n x M
// matrix of counts / (4 S) of the FP64 form, then that of the FP32 form (the fixed disc + halo +
// Long-Murali layout where the model is that layout), as doubles.
#include "bs3_host.h"

#include <cstdio>
#include <vector>

using namespace sw;

static void euler(double a, double b, double g, double R[9])
{
    const double A[9] = {cos(a), -sin(a), 0, sin(a), cos(a), 0, 0, 0, 1};
    const double B[9] = {1, 0, 0, 0, cos(b), -sin(b), 0, sin(b), cos(b)};
    const double C[9] = {cos(g), -sin(g), 0, sin(g), cos(g), 0, 0, 0, 1};
    double T_[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += B[3 * i + k] * A[3 * k + j];
            T_[3 * i + j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += C[3 * i + k] * T_[3 * k + j];
            R[3 * i + j] = s;
        }
}

template <typename T, int POT>
static std::vector<double> run(const double* P, const double* Gd, const std::vector<double>& ics, int64_t n)
{
    const int64_t nsteps = (int64_t)P[14];
    FieldT<T> fl{};
    fl.has_disc = P[0] > 0; fl.gm_disc = (T)(SW_G * P[0]); fl.disc_a = (T)P[1]; fl.disc_b2 = (T)(P[2] * P[2]);
    fl.has_halo = P[3] > 0; fl.gm_halo = (T)(SW_G * P[3]); fl.halo_rs = (T)P[4]; fl.halo_inv_rs = (T)(1.0 / P[4]);
    fl.has_bar = P[5] > 0; fl.k_bar = P[5] > 0 ? (T)(SW_G * P[5] / (2 * P[6])) : T(0); fl.bar_L = (T)P[6];
    fl.bar_a = (T)P[7]; fl.bar_b2 = (T)(P[8] * P[8]);
    GridT<T> g{};
    double R[9];
    euler(P[11], P[10], 0.0, R);
    for (int k = 0; k < 9; ++k) g.R[k] = (T)R[k];
    const int nx = (int)Gd[0], ny = (int)Gd[1], nv = (int)Gd[3], nR = (int)Gd[5], nphi = (int)Gd[6], nz = (int)Gd[7];
    const double pix = Gd[2], vmax = Gd[4];
    g.nx = nx; g.ny = ny; g.x0 = (T)(-0.5 * nx * pix); g.y0 = (T)(-0.5 * ny * pix); g.dx = g.dy = (T)pix;
    g.inv_dx = g.inv_dy = (T)(1 / pix);
    g.nv = nv; g.v0 = (T)(-vmax); g.dv = (T)(2 * vmax / nv); g.inv_dv = (T)(nv / (2 * vmax));
    g.nR = nR; g.nphi = nphi; g.nz = nz;
    const double dR = Gd[8] / nR, dphi = 2 * 3.14159265358979323846 / nphi, dz = (Gd[10] - Gd[9]) / nz;
    g.dR = (T)dR; g.inv_dR = (T)(1 / dR); g.dphi = (T)dphi; g.inv_dphi = (T)(1 / dphi); g.zmin = (T)Gd[9];
    g.dz = (T)dz; g.inv_dz = (T)(1 / dz);
    g.gh = 0; g.ncopy = 4; g.sym = 1;   // pixel and velocity grids centred on 0
    g.nd = (int64_t)nR * nphi * nz; g.npix = (int64_t)nx * ny; g.M = g.nd + g.npix + g.npix * nv;
    std::vector<T> cs(2 * (nsteps + 1));
    for (int64_t k = 0; k <= nsteps; ++k) {
        const double th = P[9] * ((double)k * P[12]);
        cs[2 * k] = (T)cos(th);
        cs[2 * k + 1] = (T)sin(th);
    }
    ModelT<T> m{};
    m.f = fl; m.g = g; m.dt = (T)P[12]; m.half_dt = (T)(0.5 * P[12]); m.omega = (T)P[9]; m.cs = cs.data();
    m.sign = 1;
    // the state as k_ics_soa lays it out: rows 0-5 the working precision, rows 6-11 (FP32) the residuals
    const int rows = sizeof(T) == 4 ? 12 : 6;
    std::vector<T> soa(rows * n);
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 6; ++k) {
            const double v = ics[6 * i + k];
            const T hi = (T)v;
            soa[k * n + i] = hi;
            if (sizeof(T) == 4) soa[(6 + k) * n + i] = (T)(v - (double)hi);
        }
    std::vector<CountT<T>> cnt((size_t)g.M * n, 0);
    std::vector<double> out((size_t)g.M * n);
    for (int64_t i = 0; i < n; ++i) {
        double worst = 0.0;
        int st = 0;
        orbit_body<T, false, true, POT>(m, soa.data(), n, i, cnt.data() + (size_t)i * g.M, nsteps, 8, worst, st);
        for (int64_t r = 0; r < g.M; ++r)
            out[(size_t)i * g.M + r] = (double)cnt[(size_t)i * g.M + r] / (4.0 * (double)nsteps);
    }
    return out;
}

int main(int argc, char** argv)
{
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 3;
    double P[16], Gd[12];
    if (fread(P, sizeof(double), 16, f) != 16 || fread(Gd, sizeof(double), 12, f) != 12) return 4;
    const int64_t n = (int64_t)P[15];
    std::vector<double> ics(6 * n);
    if (fread(ics.data(), sizeof(double), 6 * n, f) != (size_t)(6 * n)) return 5;
    fclose(f);
    const std::vector<double> u64 = run<double, POT_ANY>(P, Gd, ics, n);
    const bool dhl = P[0] > 0 && P[3] > 0 && P[5] > 0;
    const std::vector<double> u32 = dhl ? run<float, POT_DHL>(P, Gd, ics, n) : run<float, POT_ANY>(P, Gd, ics, n);
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 6;
    fwrite(u64.data(), sizeof(double), u64.size(), o);
    fwrite(u32.data(), sizeof(double), u32.size(), o);
    fclose(o);
    return 0;
}
