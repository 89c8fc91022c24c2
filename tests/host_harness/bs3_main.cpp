// Host driver for the adaptive-integrator device functions of k_orbit.cu, compiled
// for the CPU (FP64 form) so that their arithmetic can be compared with the oracle
// without a GPU.  Input file: 16 model scalars, 12 grid scalars (the last one 1 for
// Gauss-Hermite rows), n x 6 initial conditions and, in GH mode, npix x 2 reference
// (v0, s) (doubles); output: the n x M orbit matrix and the n integration times.
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

int main(int argc, char** argv)
{
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 3;
    double P[16], Gd[12];
    if (fread(P, sizeof(double), 16, f) != 16 || fread(Gd, sizeof(double), 12, f) != 12) return 4;
    const int64_t nsteps = (int64_t)P[14], n = (int64_t)P[15];
    const bool gh = Gd[11] != 0.0;
    std::vector<double> ics(6 * n);
    if (fread(ics.data(), sizeof(double), 6 * n, f) != (size_t)(6 * n)) return 5;
    const int64_t npix = (int64_t)Gd[0] * (int64_t)Gd[1];
    std::vector<double> v0s(gh ? 2 * npix : 0), tab(gh ? 2 * npix : 0);
    if (gh && fread(v0s.data(), sizeof(double), 2 * npix, f) != (size_t)(2 * npix)) return 7;
    for (int64_t q = 0; gh && q < npix; ++q) { tab[2 * q] = v0s[2 * q]; tab[2 * q + 1] = 1.0 / v0s[2 * q + 1]; }
    fclose(f);
    // model constants as the library sets them (disc, NFW from M_DM and R_s, bar)
    FieldT<double> fl{};
    fl.has_disc = P[0] > 0; fl.gm_disc = SW_G * P[0]; fl.disc_a = P[1]; fl.disc_b2 = P[2] * P[2];
    fl.has_halo = P[3] > 0; fl.gm_halo = SW_G * P[3]; fl.halo_rs = P[4]; fl.halo_inv_rs = 1.0 / P[4];
    fl.has_bar = P[5] > 0; fl.k_bar = P[5] > 0 ? SW_G * P[5] / (2 * P[6]) : 0; fl.bar_L = P[6]; fl.bar_a = P[7];
    fl.bar_b2 = P[8] * P[8];
    GridT<double> g{};
    double R[9];
    euler(P[11], P[10], 0.0, R);
    for (int k = 0; k < 9; ++k) g.R[k] = R[k];
    const int nx = (int)Gd[0], ny = (int)Gd[1], nv = (int)Gd[3], nR = (int)Gd[5], nphi = (int)Gd[6], nz = (int)Gd[7];
    const double pix = Gd[2], vmax = Gd[4];
    g.nx = nx; g.ny = ny; g.x0 = -0.5 * nx * pix; g.y0 = -0.5 * ny * pix; g.dx = g.dy = pix;
    g.inv_dx = g.inv_dy = 1 / pix;
    g.nv = gh ? 0 : nv; g.v0 = gh ? 0.0 : -vmax; g.dv = gh ? 1.0 : 2 * vmax / nv; g.inv_dv = 1 / g.dv;
    g.nR = nR; g.nphi = nphi; g.nz = nz;
    const double dR = Gd[8] / nR, dphi = 2 * 3.14159265358979323846 / nphi, dz = (Gd[10] - Gd[9]) / nz;
    g.dR = dR; g.inv_dR = 1 / dR; g.dphi = dphi; g.inv_dphi = 1 / dphi; g.zmin = Gd[9]; g.dz = dz; g.inv_dz = 1 / dz;
    g.gh = gh ? 1 : 0; g.ncopy = 4;
    g.nd = (int64_t)nR * nphi * nz; g.npix = (int64_t)nx * ny; g.M = g.nd + g.npix + (gh ? 4 * g.npix : g.npix * nv);
    ModelT<double> m{};
    m.f = fl; m.g = g; m.dt = P[12]; m.half_dt = 0.5 * P[12]; m.omega = P[9];
    m.gh_v0s = gh ? tab.data() : nullptr;
    std::vector<double> soa(6 * n), U((size_t)g.M * n, 0.0), tt(n), dr(n);
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 6; ++k) soa[k * n + i] = ics[6 * i + k];
    m.U = U.data(); m.n_orb = n; m.orbit_base = 0; m.ldu = g.M;
    for (int64_t i = 0; i < n; ++i) {
        double* col = U.data() + (size_t)i * g.M;
        int st = 0;
        if (gh) orbit_body_bs3<double, true>(m, soa.data(), n, i, col, nsteps, 1, P[13], dr[i], st, tt[i]);
        else orbit_body_bs3<double, false>(m, soa.data(), n, i, col, nsteps, 1, P[13], dr[i], st, tt[i]);
        const double s = st == ST_OK ? 1.0 / (4.0 * tt[i]) : 0.0;     // the finalisation of k_finalize_w
        for (int64_t r = 0; r < g.M; ++r) col[r] *= s;
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 6;
    fwrite(U.data(), sizeof(double), U.size(), o);
    fwrite(tt.data(), sizeof(double), n, o);
    fclose(o);
    return 0;
}
