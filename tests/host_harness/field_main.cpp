// Host driver for the force-field device functions of k_orbit.cu (disc, halo and either
// bar), compiled for the CPU in both precisions so that the arithmetic of the paper's
// Dehnen-Aly bar can be compared with the oracle without a GPU.  Input file: 10 model
// scalars (disc M, a, b; M_DM, R_s; bar M, L, b, c; bar_kind), the 8-point Gauss-Legendre
// rule's 4 positive nodes and 4 weights, n, then n x 3 bar-frame points (doubles).
// Output: for FP64, FP32 and the FP32 kernels' fixed layout (FP32 again where the model is not
// disc + halo + Long-Murali bar), phi (n) and acceleration (n x 3), as doubles.
#include "bs3_host.h"

#include <cstdio>
#include <vector>

using namespace sw;

template <typename T>
static FieldT<T> make(const double* P, const double* gl)
{
    FieldT<T> f{};
    f.has_disc = P[0] > 0; f.gm_disc = (T)(SW_G * P[0]); f.disc_a = (T)P[1]; f.disc_b2 = (T)(P[2] * P[2]);
    f.has_halo = P[3] > 0; f.gm_halo = (T)(SW_G * P[3]); f.halo_rs = (T)P[4]; f.halo_inv_rs = (T)(1.0 / P[4]);
    f.has_bar = P[5] > 0; f.k_bar = P[5] > 0 ? (T)(SW_G * P[5] / (2 * P[6])) : T(0); f.bar_L = (T)P[6];
    f.bar_a = (T)P[7]; f.bar_b2 = (T)(P[8] * P[8]);
    f.bar_kind = (int)P[9];
    f.da_gm1 = (T)(SW_G * 0.5 * P[5]); f.da_a1 = (T)(P[6] / 5.0); f.da_b1sq = (T)(P[2] * P[2]); f.da_L1 = (T)P[6];
    f.da_gm2 = (T)(SW_G * 0.5 * P[5]); f.da_a2 = (T)0.5; f.da_b2sq = (T)0.25; f.da_L2 = (T)0.1;
    for (int k = 0; k < 4; ++k) { f.gl_x[k] = (T)gl[k]; f.gl_w[k] = (T)gl[4 + k]; }
    return f;
}

template <typename T, int POT = POT_ANY>
static void eval(const FieldT<T>& f, const std::vector<double>& xyz, int64_t n, FILE* out)
{
    std::vector<double> phi(n), acc(3 * n);
    for (int64_t i = 0; i < n; ++i) {
        T ax, ay, az, ph, xb, yb;
        field<T, POT>(f, T(1), T(0), (T)xyz[3 * i], (T)xyz[3 * i + 1], (T)xyz[3 * i + 2], ax, ay, az, ph, true, xb,
                      yb);
        phi[i] = ph; acc[3 * i] = ax; acc[3 * i + 1] = ay; acc[3 * i + 2] = az;
    }
    fwrite(phi.data(), sizeof(double), n, out);
    fwrite(acc.data(), sizeof(double), 3 * n, out);
}

int main(int argc, char** argv)
{
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 3;
    double P[10], gl[8], nd;
    if (fread(P, sizeof(double), 10, f) != 10 || fread(gl, sizeof(double), 8, f) != 8 ||
        fread(&nd, sizeof(double), 1, f) != 1)
        return 4;
    const int64_t n = (int64_t)nd;
    std::vector<double> xyz(3 * n);
    if (fread(xyz.data(), sizeof(double), 3 * n, f) != (size_t)(3 * n)) return 5;
    fclose(f);
    FILE* out = fopen(argv[2], "wb");
    if (!out) return 6;
    eval<double>(make<double>(P, gl), xyz, n, out);
    eval<float>(make<float>(P, gl), xyz, n, out);
    // the fixed disc + halo + Long-Murali layout of the FP32 kernels, where the model is that layout
    const FieldT<float> f32 = make<float>(P, gl);
    if (f32.has_disc && f32.has_halo && f32.has_bar && f32.bar_kind == 0)
        eval<float, POT_DHL>(f32, xyz, n, out);
    else
        eval<float>(f32, xyz, n, out);
    fclose(out);
    return 0;
}
