// Cholesky factor L of the shifted passive Gram (in place, lower) and the explicit
// inverse X = L^{-1}: the preconditioner of the weight solve's reduced systems
// (Sec. 2.3).  Blocked right-looking in 128-wide steps; at step k
//
//   1. k_diag128 (one CTA): L_kk = chol(A_kk) and D_k = L_kk^{-1}, blocked by
//      32 in shared memory: one warp factors and inverts each 32 x 32 diagonal
//      sub-block in registers while the other warps assemble the inverse's
//      earlier block rows; panels and trailing updates use all threads;
//   2. k_panel128: the panel below, L_ik = A_ik D_k^T (FP32, in place), also
//      written as BF16 hi + lo halves (the split operand of step 3);
//   3. k_tc_sub<lower>: the trailing update A_ij -= L_ik L_jk^T on the 5th-
//      generation tensor cores: the tile is accumulated in TMEM from the three
//      leading products of the split (hi hi, hi lo, lo hi; ~2^-16 relative)
//      and subtracted from the FP32 trailing matrix in the epilogue;
//   4. k_trmm128: block row k of the inverse, X_k <- D_k X_k (FP32), also
//      written transposed as BF16 hi + lo halves;
//   5. k_tc_sub<full>: the rows below, X_i -= L_ik X_k (tensor cores).
//
// Steps 1, 2 and 4 are FP32 SIMT; 3 and 5 hold the O(K^3) work.  The split
// products make the factor a preconditioner accurate to ~1e-4 relative, which
// the conjugate-gradient solve that uses it absorbs in one or two extra steps.
#include "sw_linalg.cuh"
#include "sw_tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

namespace sw {

namespace ctc {

using namespace sw::tc;

constexpr int DB = 128;  // block width
constexpr int LP = DB + 1;

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// eight FP32 values as their BF16 hi and lo halves, 16 bytes each (element 2q in the low half of word q)
__device__ __forceinline__ void split8(const float (&v)[8], uint4& h, uint4& l)
{
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * q] - __low2float(hh), v[2 * q + 1] - __high2float(hh));
        hw[q] = (uint32_t)__bfloat16_as_ushort(hh.x) | ((uint32_t)__bfloat16_as_ushort(hh.y) << 16);
        lw[q] = (uint32_t)__bfloat16_as_ushort(ll.x) | ((uint32_t)__bfloat16_as_ushort(ll.y) << 16);
    }
    h = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    l = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// byte offset of the 16-byte chunk j (elements 8 j .. 8 j + 7) of row r in a 128 x 64 BF16 box with the
// 128-byte swizzle (the layout a TMA load with that swizzle produces, which the UMMA descriptor reads)
__device__ __forceinline__ int sw128_off(int r, int j) { return r * 128 + ((j ^ (r & 7)) << 4); }

// ---------------------------------------------------------------------------
// 1. Diagonal block: Cholesky and triangular inverse, blocked by 32 inside the
// CTA (256 threads).  The block sits in shared memory (A, row pitch AP; rows
// and columns beyond bs are an identity, so a short last block needs no
// special case).  For each 32-wide sub-block s, with the rows below it R_s:
//   A. warp 0 factors the diagonal sub-block L_ss, one row per lane in
//      registers: the pivot of column j + 1 is formed by its own lane and
//      broadcast by one shuffle, the next two columns are updated through
//      shuffles and the rest through the transposed column buffer CT.
//      Meanwhile warps 1-7 apply the part of the previous step's trailing
//      update that the next steps need last (columns beyond sub-block s + 1)
//      and advance the inverse (below);
//   B. one thread per row of R_s solves L_is L_ss^T = A_is by forward
//      substitution (warps 1-3), while warp 0 inverts L_ss (one column of
//      X_ss per lane);
//   C. all threads update column block s + 1 by the new panel.
// The inverse X = L^{-1} below the diagonal, by block rows r: T_j = sum_{k=j}
// ^{r-1} L_rk X_kj (formed while sub-block r is factored) and X_rj = -X_rr T_j
// (formed while sub-block r + 1 is factored; the last block row at the end).
// Every register index is static (the 32-step loops are unrolled).
// ---------------------------------------------------------------------------
constexpr int DIAG_THREADS = 256;
constexpr int AP = DB + 4;    // row pitch: 16-byte rows, consecutive rows in distinct bank groups
constexpr int SB = 32;        // sub-block width
constexpr int CTP = SB + 4;   // pitch of the 32-wide buffers
constexpr int TBUF = 3 * SB * CTP;

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float dot4(float4 a, float4 b, float acc)
{
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, acc))));
}

// T_j = sum_{k=j}^{r-1} L_rk X_kj for j < r into Tb: 4 x 4 tiles, tile q = (j, ta, tb) with rows
// 4 ta .. 4 ta + 3 and columns 4 tb .. 4 tb + 3 of T_j (consecutive q: consecutive tb, so the
// rows of X are read by eight threads at distinct 16-byte chunks and the rows of L are shared)
__device__ __forceinline__ void inverse_t_part(const float* __restrict__ A, const float* __restrict__ X,
                                               float* __restrict__ Tb, int r, int tid, int NT)
{
    for (int q = tid; q < 64 * r; q += NT) {
        const int j = q >> 6, ta = (q >> 3) & 7, tb = q & 7;
        const float* pr = A + (SB * r + 4 * ta) * AP;
        const float* xc = X + SB * j + 4 * tb;
        float acc[4][4] = {};
#pragma unroll 2
        for (int c = SB * j; c < SB * r; c += 4) {
            float4 p[4], x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) p[u] = ld4(pr + u * AP + c);
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = ld4(xc + (c + u) * AP);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float pv[4] = {p[u].x, p[u].y, p[u].z, p[u].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    acc[u][0] = fmaf(pv[k], x[k].x, acc[u][0]);
                    acc[u][1] = fmaf(pv[k], x[k].y, acc[u][1]);
                    acc[u][2] = fmaf(pv[k], x[k].z, acc[u][2]);
                    acc[u][3] = fmaf(pv[k], x[k].w, acc[u][3]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            *reinterpret_cast<float4*>(Tb + (j * SB + 4 * ta + u) * CTP + 4 * tb) =
                make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    }
}

// X_rj = -X_rr T_j for j < r (X_rr lower triangular: columns c <= row), 4 x 4 tiles as above
__device__ __forceinline__ void inverse_x_part(float* __restrict__ X, const float* __restrict__ Tb, int r, int tid,
                                               int NT)
{
    for (int q = tid; q < 64 * r; q += NT) {
        const int j = q >> 6, ta = (q >> 3) & 7, tb = q & 7;
        const float* xr = X + (SB * r + 4 * ta) * AP + SB * r;
        const float* tj = Tb + j * SB * CTP + 4 * tb;
        float acc[4][4] = {};
        for (int c = 0; c <= 4 * ta; c += 4) {
            float4 p[4], t4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) p[u] = ld4(xr + u * AP + c);
#pragma unroll
            for (int u = 0; u < 4; ++u) t4[u] = ld4(tj + (c + u) * CTP);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float pv[4] = {p[u].x, p[u].y, p[u].z, p[u].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    acc[u][0] = fmaf(pv[k], t4[k].x, acc[u][0]);
                    acc[u][1] = fmaf(pv[k], t4[k].y, acc[u][1]);
                    acc[u][2] = fmaf(pv[k], t4[k].z, acc[u][2]);
                    acc[u][3] = fmaf(pv[k], t4[k].w, acc[u][3]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            *reinterpret_cast<float4*>(X + (SB * r + 4 * ta + u) * AP + SB * j + 4 * tb) =
                make_float4(-acc[u][0], -acc[u][1], -acc[u][2], -acc[u][3]);
    }
}

// A[i][j] -= sum_k A[i][p0 + k] A[j][p0 + k] over the lower 4 x 4 tiles of rows and columns r0 .. 127
__device__ __forceinline__ void trailing_rest(float* __restrict__ A, int p0, int r0, int tid, int NT)
{
    const int nt = (DB - r0) >> 2;
    for (int q = tid; q < nt * nt; q += NT) {
        const int ti = q / nt, tj = q - ti * nt;
        if (tj > ti) continue;
        const float* ra = A + (r0 + 4 * ti) * AP + p0;
        const float* rb = A + (r0 + 4 * tj) * AP + p0;
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
#pragma unroll 2
        for (int k = 0; k < SB; k += 4) {
            float4 u[4], v[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) u[r] = ld4(ra + r * AP + k);
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = ld4(rb + c * AP + k);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = dot4(u[r], v[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float4* o = reinterpret_cast<float4*>(A + (r0 + 4 * ti + r) * AP + r0 + 4 * tj);
            float4 v = *o;
            v.x -= acc[r][0]; v.y -= acc[r][1]; v.z -= acc[r][2]; v.w -= acc[r][3];
            *o = v;
        }
    }
}

// Phase A of k_diag128 for warp 0: Cholesky of the 32 x 32 diagonal sub-block at (c0, c0), one row per
// lane in registers; writes L_ss back into A (upper part zero), its columns into CT and 1 / L_jj into RR.
// Kept out of line so that its registers are allocated apart from the rest of the kernel.
__device__ __noinline__ void warp_factor32(float* __restrict__ A, float* __restrict__ CT, float* __restrict__ RR,
                                           int c0, int bs, int64_t j0, int* info, int lane)
{
    float a[SB];
#pragma unroll
    for (int k = 0; k < SB; k += 4) {
        const float4 v = ld4(A + (c0 + lane) * AP + c0 + k);
        a[k] = v.x; a[k + 1] = v.y; a[k + 2] = v.z; a[k + 3] = v.w;
    }
    float d = __shfl_sync(0xffffffffu, a[0], 0);
    float rmine = 0.f;   // 1 / L_jj of this lane's column j = lane
    int bad = 0;         // first non-positive pivot of the sub-block, plus one
#pragma unroll
    for (int j = 0; j < SB; ++j) {
        const bool ok = d > 0.f;
        bad = (!ok && bad == 0 && c0 + j < bs) ? j + 1 : bad;
        const float r = rsqrtf(ok ? d : 1e-30f);
        rmine = lane == j ? r : rmine;
        const float lij = lane >= j ? a[j] * r : 0.f;
        a[j] = lij;
        CT[j * CTP + lane] = lij;
        if (j + 1 < SB) {
            // the next pivot: lane j + 1 subtracts its own l_(j+1) j^2, one shuffle broadcasts it
            const float dn = a[j + 1] - lij * lij;
            d = __shfl_sync(0xffffffffu, dn, j + 1 < SB ? j + 1 : 0);
        }
        // the rest of column j reaches every lane as broadcast reads of its row of CT
        __syncwarp();
#pragma unroll
        for (int k4 = ((j + 1) & ~3); k4 < SB; k4 += 4) {
            const float4 c = ld4(CT + j * CTP + k4);
            if (k4 + 0 > j) a[k4 + 0] -= lij * c.x;
            if (k4 + 1 > j) a[k4 + 1] -= lij * c.y;
            if (k4 + 2 > j) a[k4 + 2] -= lij * c.z;
            if (k4 + 3 > j) a[k4 + 3] -= lij * c.w;
        }
    }
    RR[lane] = rmine;
    if (bad && lane == 0 && info) atomicCAS(info, 0, (int)(j0 + c0 + bad));
#pragma unroll
    for (int k = 0; k < SB; k += 4)
        *reinterpret_cast<float4*>(A + (c0 + lane) * AP + c0 + k) =
            make_float4(k <= lane ? a[k] : 0.f, k + 1 <= lane ? a[k + 1] : 0.f,
                        k + 2 <= lane ? a[k + 2] : 0.f, k + 3 <= lane ? a[k + 3] : 0.f);
}

__global__ void __launch_bounds__(DIAG_THREADS, 1) k_diag128(float* __restrict__ G, int64_t ld, int64_t j0, int bs,
                                                             float* __restrict__ D /* D_k^T */, int* info,
                                                             int write_L, uint4* __restrict__ Dsw)
{
    extern __shared__ __align__(16) float sm[];
    float* A = sm;                  // DB x AP: the block, then L
    float* X = A + DB * AP;         // DB x AP: L^{-1}
    float* CT = X + DB * AP;        // SB x CTP: CT[j][i] = L(c0 + i, c0 + j) of the current sub-block
    float* Tb = CT + SB * CTP;      // 2 x TBUF: the sums T_j of an inverse block row, by parity of r
    float* RR = Tb + 2 * TBUF;      // SB: 1 / L_jj of the current sub-block
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // the panel kernel that follows may start now: it stages its rows of A (final before this
    // kernel began) and waits for this grid's D before reading it
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // ---- load the lower triangle (16-byte chunks that reach it; the rest of A is never read), all
    // in flight; rows beyond bs are the identity; X = 0
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        float4 v[8];
#pragma unroll
        for (int uu = 0; uu < 8; ++uu) {
            const int u = 8 * half + uu;
            const int e = t + DIAG_THREADS * u, i = e >> 5, l4 = (e & 31) * 4;
            const float* g = G + (size_t)(j0 + i) * ld + j0 + l4;
            if (l4 > i) continue;
            if (i < bs && l4 + 3 < bs) {
                v[uu] = ld4(g);
            } else {
                float w[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) w[c] = (i < bs && l4 + c < bs) ? g[c] : (i == l4 + c ? 1.f : 0.f);
                v[uu] = make_float4(w[0], w[1], w[2], w[3]);
            }
        }
#pragma unroll
        for (int uu = 0; uu < 8; ++uu) {
            const int u = 8 * half + uu;
            const int e = t + DIAG_THREADS * u, i = e >> 5, l4 = (e & 31) * 4;
            if (l4 <= i) *reinterpret_cast<float4*>(A + i * AP + l4) = v[uu];
            *reinterpret_cast<float4*>(X + i * AP + l4) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int s = 0; s < DB / SB; ++s) {
        const int c0 = SB * s;
        // ======== A
        if (warp == 0) {
            warp_factor32(A, CT, RR, c0, bs, j0, info, lane);
        } else if (warp != 4) {
            // warps 1-3 and 5-7 (warp 4 shares warp 0's scheduler and stays idle)
            const int tid = t - (warp < 4 ? 32 : 64), NT = DIAG_THREADS - 64;
            auto bar = [] { asm volatile("bar.sync 1, %0;" ::"n"(DIAG_THREADS - 64) : "memory"); };
            // the previous panel's update of columns beyond sub-block s + 1 (columns of s + 1 were done in C)
            if (s >= 1 && s <= 2) trailing_rest(A, c0 - SB, c0 + SB, tid, NT);
            // X_(s-1) j = -X_(s-1)(s-1) T_j, then T_j of block row s (it needs block row s - 1)
            if (s >= 2) {
                inverse_x_part(X, Tb + ((s - 1) & 1) * TBUF, s - 1, tid, NT);
                bar();
            }
            if (s >= 1) inverse_t_part(A, X, Tb + (s & 1) * TBUF, s, tid, NT);
        }
        __syncthreads();
        // ======== B
        if (warp == 0) {
            // X_ss = L_ss^{-1}, lane l holds column l
            float x[SB], rr[SB];
#pragma unroll
            for (int i = 0; i < SB; i += 4) {
                const float4 v = ld4(RR + i);
                rr[i] = v.x; rr[i + 1] = v.y; rr[i + 2] = v.z; rr[i + 3] = v.w;
            }
#pragma unroll
            for (int i = 0; i < SB; ++i) x[i] = i == lane ? 1.f : 0.f;
#pragma unroll
            for (int k = 0; k < SB; ++k) {
                x[k] *= rr[k];
#pragma unroll
                for (int i4 = ((k + 1) & ~3); i4 < SB; i4 += 4) {
                    const float4 c = ld4(CT + k * CTP + i4);
                    if (i4 + 0 > k) x[i4 + 0] -= c.x * x[k];
                    if (i4 + 1 > k) x[i4 + 1] -= c.y * x[k];
                    if (i4 + 2 > k) x[i4 + 2] -= c.z * x[k];
                    if (i4 + 3 > k) x[i4 + 3] -= c.w * x[k];
                }
            }
#pragma unroll
            for (int i = 0; i < SB; ++i) X[(c0 + i) * AP + c0 + lane] = x[i];
        } else if (t - 32 < DB - c0 - SB) {
            // row i of the panel: y L_ss^T = a_i by forward substitution
            const int i = c0 + SB + (t - 32);
            float y[SB], rr[SB];
#pragma unroll
            for (int k = 0; k < SB; k += 4) {
                const float4 v = ld4(A + i * AP + c0 + k);
                y[k] = v.x; y[k + 1] = v.y; y[k + 2] = v.z; y[k + 3] = v.w;
                const float4 w = ld4(RR + k);
                rr[k] = w.x; rr[k + 1] = w.y; rr[k + 2] = w.z; rr[k + 3] = w.w;
            }
#pragma unroll
            for (int k = 0; k < SB; ++k) {
                y[k] *= rr[k];
#pragma unroll
                for (int j4 = ((k + 1) & ~3); j4 < SB; j4 += 4) {
                    const float4 c = ld4(CT + k * CTP + j4);
                    if (j4 + 0 > k) y[j4 + 0] -= c.x * y[k];
                    if (j4 + 1 > k) y[j4 + 1] -= c.y * y[k];
                    if (j4 + 2 > k) y[j4 + 2] -= c.z * y[k];
                    if (j4 + 3 > k) y[j4 + 3] -= c.w * y[k];
                }
            }
#pragma unroll
            for (int k = 0; k < SB; k += 4)
                *reinterpret_cast<float4*>(A + i * AP + c0 + k) = make_float4(y[k], y[k + 1], y[k + 2], y[k + 3]);
        }
        __syncthreads();
        if (s == DB / SB - 1) break;
        // ======== C: column block s + 1 -= panel (rows c0 + 32 .. 127); thread (cg, rs) = (t % 8, t / 8)
        // forms columns c0 + 32 + cg + 8 jj of rows c0 + 32 + rs + 32 rr
        {
            const int cg = t & 7, rs = t >> 3, nrb = 3 - s, c1 = c0 + SB;
            float acc[3][4];
#pragma unroll
            for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[rr][jj] = 0.f;
#pragma unroll 2
            for (int k = 0; k < SB; k += 4) {
                float4 xv[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) xv[jj] = ld4(A + (c1 + cg + 8 * jj) * AP + c0 + k);
#pragma unroll
                for (int rr = 0; rr < 3; ++rr) {
                    if (rr < nrb) {
                        const float4 av = ld4(A + (c1 + rs + SB * rr) * AP + c0 + k);
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) acc[rr][jj] = dot4(av, xv[jj], acc[rr][jj]);
                    }
                }
            }
#pragma unroll
            for (int rr = 0; rr < 3; ++rr)
                if (rr < nrb) {
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) A[(c1 + rs + SB * rr) * AP + c1 + cg + 8 * jj] -= acc[rr][jj];
                }
        }
        __syncthreads();
    }
    // ---- the last block row of the inverse (its sums were formed while sub-block 3 was factored)
    inverse_x_part(X, Tb + ((DB / SB - 1) & 1) * TBUF, DB / SB - 1, t, DIAG_THREADS);
    __syncthreads();
    // ---- L back into G when asked (lower triangle of the block, 16-byte stores where the chunk lies in
    // it; the factorisation itself needs only D and the panels)
    if (write_L) {
#pragma unroll 4
        for (int u = 0; u < 16; ++u) {
            const int e = t + DIAG_THREADS * u, i = e >> 5, l4 = (e & 31) * 4;
            if (i >= bs || l4 > i) continue;
            float* g = G + (size_t)(j0 + i) * ld + j0 + l4;
            const float4 v = ld4(A + i * AP + l4);
            if (l4 + 3 <= i && l4 + 3 < bs) {
                *reinterpret_cast<float4*>(g) = v;
            } else {
                const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (l4 + c <= i && l4 + c < bs) g[c] = w[c];
            }
        }
    }
    // D transposed, Dt[l][c] = D[c][l] (zero outside c < bs, l <= c): thread (c, half) reads rows of X as
    // 16-byte vectors and writes four rows of Dt, each write coalesced over c.  Groups of four rows
    // wholly above the diagonal (l4 > c) are not written: the readers take them as zero
    {
        const int c = t & (DB - 1), h = t >> 7;
        const bool cin = c < bs;
#pragma unroll 4
        for (int l4 = 4 * h; l4 < DB; l4 += 8) {
            if (l4 > c) continue;
            const float4 v = ld4(X + c * AP + l4);
            D[(l4 + 0) * DB + c] = cin && l4 + 0 <= c ? v.x : 0.f;
            D[(l4 + 1) * DB + c] = cin && l4 + 1 <= c ? v.y : 0.f;
            D[(l4 + 2) * DB + c] = cin && l4 + 2 <= c ? v.z : 0.f;
            D[(l4 + 3) * DB + c] = cin && l4 + 3 <= c ? v.w : 0.f;
        }
    }
    // D as the tensor-core panel's B operand (Dsw non-NULL): the BF16 hi and lo halves of D[c][l] (zero
    // for l > c or c >= bs), rows c, in four 128 x 64 boxes of 16 KB -- hi l < 64, hi l >= 64, lo l < 64,
    // lo l >= 64 -- in the 128-byte-swizzled layout, so that one flat copy puts them in shared memory
    if (Dsw) {
#pragma unroll 2
        for (int u = t; u < DB * 16; u += DIAG_THREADS) {
            const int c = u >> 4, j16 = u & 15, b = j16 >> 3, j = j16 & 7, l0 = 8 * j16;
            const float4 x0 = ld4(X + c * AP + l0), x1 = ld4(X + c * AP + l0 + 4);
            const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = (c < bs && l0 + q <= c) ? xv[q] : 0.f;
            uint4 h, l;
            split8(v, h, l);
            const int off = sw128_off(c, j) >> 4;
            Dsw[b * 1024 + off] = h;
            Dsw[(2 + b) * 1024 + off] = l;
        }
    }
}

constexpr size_t DIAG_SMEM = sizeof(float) * (2 * DB * AP + SB * CTP + 2 * TBUF + SB);

// ---------------------------------------------------------------------------
// 2. Panel: P = A D^T for m rows below the diagonal block (A = G[r0 + i][j0 ..
// j0 + 127]), in place in G, and its BF16 hi + lo halves (m x 128, rows pst
// elements apart: 128, or 256 when two panels share a row).
// 32 rows per CTA of 256 threads; thread (tr, tc) = (t / 16, t % 16) computes
// rows 2 tr, 2 tr + 1 and columns 4 tc .. 4 tc + 3 and 64 + 4 tc .. 64 + 4 tc +
// 3 (two 16-byte loads of a row of D^T in distinct bank groups).  D arrives
// transposed (Dt[l][c] = D[c][l]) and is staged by 16-byte copies.
// ---------------------------------------------------------------------------
constexpr int PR = 32;
constexpr int DTP = DB + 4;   // padded row of DT (16-byte aligned, conflict-free float4 rows)
__global__ void __launch_bounds__(256) k_panel128(float* __restrict__ G, int64_t ld, int64_t j0, int64_t r0,
                                                  int64_t m, const float* __restrict__ Dt,
                                                  __nv_bfloat16* __restrict__ Ph, __nv_bfloat16* __restrict__ Pl,
                                                  int pst)
{
    extern __shared__ __align__(16) float sm[];
    float* DT = sm;              // DB x DTP
    float* As = DT + DB * DTP;   // PR x LP
    const int t = threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.x * PR;
#pragma unroll 8
    for (int e = t; e < PR * DB; e += 256) {
        const int i = e >> 7, l = e & (DB - 1);
        const int64_t gi = row0 + i;
        As[i * LP + l] = gi < m ? G[(size_t)(r0 + gi) * ld + j0 + l] : 0.f;
    }
    // D comes from the diagonal-block kernel just before this one (a no-op without a programmatic
    // launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
#pragma unroll 4
    for (int e4 = t; e4 < DB * DB / 4; e4 += 256) {
        const int l = (4 * e4) >> 7, c = (4 * e4) & (DB - 1);
        *reinterpret_cast<float4*>(DT + l * DTP + c) =
            (l & ~3) > c ? make_float4(0.f, 0.f, 0.f, 0.f) : reinterpret_cast<const float4*>(Dt)[e4];
    }
    __syncthreads();
    const int tr = t >> 4, tc = t & 15;
    float acc[2][8];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;
#pragma unroll 8
    for (int l = 0; l < DB; ++l) {
        const float a0 = As[(2 * tr) * LP + l], a1 = As[(2 * tr + 1) * LP + l];
        const float4 d0 = *reinterpret_cast<const float4*>(&DT[l * DTP + 4 * tc]);
        const float4 d1 = *reinterpret_cast<const float4*>(&DT[l * DTP + 64 + 4 * tc]);
        const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            acc[0][q] += a0 * dv[q];
            acc[1][q] += a1 * dv[q];
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int64_t gi = row0 + 2 * tr + r;
        if (gi >= m) continue;
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            const int c = 64 * hf + 4 * tc;
            const float* v = &acc[r][4 * hf];
            *reinterpret_cast<float4*>(G + (size_t)(r0 + gi) * ld + j0 + c) = make_float4(v[0], v[1], v[2], v[3]);
            uint32_t hw[2], lw[2];
#pragma unroll
            for (int q = 0; q < 4; q += 2) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(v[q], v[q + 1]);
                const __nv_bfloat162 lo = __floats2bfloat162_rn(v[q] - __low2float(h), v[q + 1] - __high2float(h));
                hw[q / 2] = (uint32_t)__bfloat16_as_ushort(h.x) | ((uint32_t)__bfloat16_as_ushort(h.y) << 16);
                lw[q / 2] = (uint32_t)__bfloat16_as_ushort(lo.x) | ((uint32_t)__bfloat16_as_ushort(lo.y) << 16);
            }
            *reinterpret_cast<uint2*>(Ph + (size_t)gi * pst + c) = make_uint2(hw[0], hw[1]);
            *reinterpret_cast<uint2*>(Pl + (size_t)gi * pst + c) = make_uint2(lw[0], lw[1]);
        }
    }
}

constexpr size_t PANEL_SMEM = sizeof(float) * (PR * LP + DB * DTP);

// ---------------------------------------------------------------------------
// 2'. Panel on the tensor cores: the same P = A D^T, one 128-row tile per CTA of 128
// threads.  The CTA splits its rows of A (FP32, final before the diagonal block began,
// so staged before the programmatic wait) into BF16 hi + lo halves in the 128-byte-
// swizzled K-major layout, copies the diagonal kernel's split D (Dsw) in one bulk copy,
// and one thread issues the three leading products of the split (hi hi, hi lo, lo hi)
// into a 128-column TMEM accumulator; each warp then drains its 32 rows, writing P in
// place into G and its own BF16 halves.  Waits are bounded: on expiry the CTA records an
// error, waits for its products once more (bounded), frees TMEM and returns.
// ---------------------------------------------------------------------------
constexpr int PT_BOX = 128 * 64 * 2;                    // one 128 x 64 BF16 box
constexpr int PT_SMEM = 8 * PT_BOX + 1024 + 64;
__global__ void __launch_bounds__(128, 1) k_panel_tc(float* __restrict__ G, int64_t ld, int64_t j0, int64_t r0,
                                                     int64_t m, const uint4* __restrict__ Dsw,
                                                     __nv_bfloat16* __restrict__ Ph, __nv_bfloat16* __restrict__ Pl,
                                                     int pst, int* err)
{
    extern __shared__ unsigned char smraw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* Ahi = base;                 // boxes: columns 0 .. 63, 64 .. 127
    unsigned char* Alo = base + 2 * PT_BOX;
    unsigned char* Bop = base + 4 * PT_BOX;    // D: hi 0 .. 63, hi 64 .. 127, lo 0 .. 63, lo 64 .. 127
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + 8 * PT_BOX);   // [0] the copy of D, [1] the products
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
    volatile int* go = reinterpret_cast<volatile int*>(tslot + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int64_t row0 = (int64_t)blockIdx.x * 128;
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // A: sixteen (row, 8-column chunk) units per thread, a warp covering two rows with 512-byte reads
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
        const int u = t + 128 * k, i = u >> 4, j16 = u & 15;
        const int64_t gi = row0 + i;
        float v[8];
        if (gi < m) {
            const float* g = G + (size_t)(r0 + gi) * ld + j0 + 8 * j16;
            const float4 a0 = *reinterpret_cast<const float4*>(g), a1 = *reinterpret_cast<const float4*>(g + 4);
            v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w; v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = 0.f;
        }
        uint4 h, l;
        split8(v, h, l);
        const int off = (j16 >> 3) * PT_BOX + sw128_off(i, j16 & 7);
        *reinterpret_cast<uint4*>(Ahi + off) = h;
        *reinterpret_cast<uint4*>(Alo + off) = l;
    }
    // D comes from the diagonal-block kernel just before this one
    asm volatile("griddepcontrol.wait;" ::: "memory");
    fence_proxy_async_smem();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (t == 0) {
        mbar_expect_tx(&bar[0], 4 * PT_BOX);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         su32(Bop)),
                     "l"((uint64_t)Dsw), "r"(4 * PT_BOX), "r"(su32(&bar[0]))
                     : "memory");
        int ok = mbar_wait(&bar[0], 0) ? 1 : 0;
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = idesc_bf16(128, 128);
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const uint64_t da = smem_desc(su32(Ahi + b * PT_BOX)), dal = smem_desc(su32(Alo + b * PT_BOX));
                const uint64_t db = smem_desc(su32(Bop + b * PT_BOX)), dbl = smem_desc(su32(Bop + (2 + b) * PT_BOX));
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    umma(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (b | k) != 0);
                    umma(tmem, da + (uint64_t)(2 * k), dbl + (uint64_t)(2 * k), idesc, 1u);
                    umma(tmem, dal + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, 1u);
                }
            }
            umma_commit(&bar[1]);
        } else {
            atomicExch(err, 1);
            mbar_wait(&bar[0], 0);   // the copy may still be in flight: one more bounded wait
        }
        *go = ok;
    }
    __syncthreads();
    if (*go) {
        if (!mbar_wait(&bar[1], 0)) {
            if (lane == 0) atomicExch(err, 1);
            mbar_wait(&bar[1], 0);   // its products still run: give them one more bounded wait
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int i = 32 * warp + lane;
            const int64_t gi = row0 + i;
#pragma unroll 1
            for (int c0 = 0; c0 < DB; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
                if (gi < m) {
                    float* g = G + (size_t)(r0 + gi) * ld + j0 + c0;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4*>(g + 4 * q) =
                            make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                        __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float f[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) f[e] = __uint_as_float(v[8 * q + e]);
                        uint4 h, l;
                        split8(f, h, l);
                        *reinterpret_cast<uint4*>(Ph + (size_t)gi * pst + c0 + 8 * q) = h;
                        *reinterpret_cast<uint4*>(Pl + (size_t)gi * pst + c0 + 8 * q) = l;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
    }
}

// ---------------------------------------------------------------------------
// 4. Block row of the inverse: X[j0 + i][c] <- sum_l D[i][l] X[j0 + l][c] for
// the ncols leading columns (in place), and its transpose as BF16 hi + lo
// halves: XT[c][i] (ncols x 128, rows xst elements apart: 128 or 256).  32 columns per CTA of 256
// threads; thread (trow, tcol) = (t / 16, t % 16) computes rows 8 trow .. 8
// trow + 7 and columns 2 tcol, 2 tcol + 1.  D arrives transposed (Dt[l][i] =
// D[i][l]) and is staged by 16-byte copies.
// ---------------------------------------------------------------------------
constexpr int TC = 32;
constexpr int SSP = TC + 4;
__global__ void __launch_bounds__(256) k_trmm128(float* __restrict__ X, int64_t ld, int64_t j0, int bs,
                                                 int64_t ncols, const float* __restrict__ Dt,
                                                 __nv_bfloat16* __restrict__ XTh, __nv_bfloat16* __restrict__ XTl,
                                                 int xst)
{
    extern __shared__ __align__(16) float sm[];
    float* DT = sm;                   // DB x DTP
    float* Ss = DT + DB * DTP;        // DB x SSP
    __nv_bfloat16* Th = reinterpret_cast<__nv_bfloat16*>(Ss + DB * SSP);   // TC x (DB + 8)
    __nv_bfloat16* Tl = Th + TC * (DB + 8);
    const int t = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * TC;
#pragma unroll 8
    for (int e = t; e < DB * TC; e += 256) {
        const int i = e / TC, cc = e % TC;
        const int64_t gc = c0 + cc;
        Ss[i * SSP + cc] = (i < bs && gc < ncols) ? X[(size_t)(j0 + i) * ld + gc] : 0.f;
    }
#pragma unroll 4
    for (int e4 = t; e4 < DB * DB / 4; e4 += 256) {
        const int l = (4 * e4) >> 7, i = (4 * e4) & (DB - 1);
        *reinterpret_cast<float4*>(DT + l * DTP + i) =
            (l & ~3) > i ? make_float4(0.f, 0.f, 0.f, 0.f) : reinterpret_cast<const float4*>(Dt)[e4];
    }
    __syncthreads();
    const int trow = t >> 4, tcol = t & 15;
    float acc[8][2];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k][0] = acc[k][1] = 0.f;
    const int lmax = 8 * trow + 7;   // D[i][l] = 0 for l > i
#pragma unroll 4
    for (int l = 0; l <= lmax; ++l) {
        const float2 sv = *reinterpret_cast<const float2*>(&Ss[l * SSP + 2 * tcol]);
        const float4 d0 = *reinterpret_cast<const float4*>(&DT[l * DTP + 8 * trow]);
        const float4 d1 = *reinterpret_cast<const float4*>(&DT[l * DTP + 8 * trow + 4]);
        const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            acc[k][0] += dv[k] * sv.x;
            acc[k][1] += dv[k] * sv.y;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = 8 * trow + k;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int cc = 2 * tcol + j;
            const int64_t gc = c0 + cc;
            if (i < bs && gc < ncols) X[(size_t)(j0 + i) * ld + gc] = acc[k][j];
            __nv_bfloat16 h, lo;
            split_bf16(i < bs ? acc[k][j] : 0.f, h, lo);
            Th[cc * (DB + 8) + i] = h;
            Tl[cc * (DB + 8) + i] = lo;
        }
    }
    __syncthreads();
    // coalesced rows of XT: 32 columns x 128 BF16 = 16 chunks of 16 bytes per row and half
    for (int e = t; e < TC * 16; e += 256) {
        const int cc = e >> 4, ch = e & 15;
        const int64_t gc = c0 + cc;
        if (gc >= ncols) continue;
        *reinterpret_cast<uint4*>(XTh + (size_t)gc * xst + ch * 8) =
            *reinterpret_cast<const uint4*>(Th + cc * (DB + 8) + ch * 8);
        *reinterpret_cast<uint4*>(XTl + (size_t)gc * xst + ch * 8) =
            *reinterpret_cast<const uint4*>(Tl + cc * (DB + 8) + ch * 8);
    }
}

constexpr size_t TRMM_SMEM = sizeof(float) * (DB * DTP + DB * SSP) + 2 * sizeof(__nv_bfloat16) * TC * (DB + 8);

// ---------------------------------------------------------------------------
// 3, 5. C[m x n] -= (A_hi + A_lo)(B_hi + B_lo)^T over a contraction of 64 nk, the
// A and B operands K-major BF16 (rows of their maps), in 128 x 128 tiles (LOWER:
// only tiles with tj <= ti), the operand rows of tile (ti, tj) starting at
// ra0 + 128 ti and rb0 + 128 tj; C is the FP32 region at (cy0, cx0) of the
// matrix behind the map mc.  Persistent: each CTA (one per SM) walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  Warp 0 issues TMA loads (128-byte
// swizzle) through a 3-stage ring; one thread of warp 1 issues tcgen05.mma into
// one of two 128-column TMEM accumulators; warps 2-5 drain the other: each
// 128 x 32 slice goes TMEM -> registers -> negated into a swizzled shared-memory
// box -> a TMA reduce-add into C, so the read-modify-write of C happens in L2
// and no thread loads C.  The epilogue's decisions are taken by one thread and
// shared through a named barrier, so its four warps never diverge.  Every wait
// is bounded: on expiry the CTA records an error, stops issuing, waits for its
// own copies and products in flight, frees TMEM and returns.
// ---------------------------------------------------------------------------
constexpr int BM = 128, BN = 128, BKC = 64;
constexpr int OP_BYTES = BM * BKC * 2;                 // one 128 x 64 BF16 operand box
constexpr int STAGES = 3, STAGE_BYTES = 4 * OP_BYTES;  // A_hi, B_hi, A_lo, B_lo
constexpr int CBOX_COLS = 32, CBOX_BYTES = BM * CBOX_COLS * 4;   // FP32 128 x 32 box of C
constexpr int SUB_SMEM = STAGES * STAGE_BYTES + 2 * CBOX_BYTES + 1024 + 256;
constexpr int SUB_THREADS = 192;
constexpr uint32_t TMEM_COLS = 256;                    // two 128-column accumulators

template <bool LOWER>
__device__ __forceinline__ void tile_of(int64_t t, int64_t tiles_n, int64_t& ti, int64_t& tj)
{
    if (LOWER) {
        ti = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        while (ti * (ti + 1) / 2 > t) --ti;
        tj = t - ti * (ti + 1) / 2;
    } else {
        ti = t / tiles_n;
        tj = t % tiles_n;
    }
}

template <bool LOWER>
__global__ void __launch_bounds__(SUB_THREADS, 1)
    k_tc_sub(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap ma_lo,
             const __grid_constant__ CUtensorMap mb, const __grid_constant__ CUtensorMap mb_lo,
             const __grid_constant__ CUtensorMap mc, int cx0, int cy0, int ra0, int rb0, int64_t n_tiles,
             int64_t tiles_n, int nk, int* err)
{
    extern __shared__ unsigned char smraw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* cstage = base + STAGES * STAGE_BYTES;   // two 1024-aligned C boxes
    uint64_t* full = reinterpret_cast<uint64_t*>(cstage + 2 * CBOX_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* epi_go = abort_flag + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        int64_t it = 0;
        for (int64_t t = blockIdx.x; t < n_tiles && !*abort_flag; t += gridDim.x) {
            int64_t ti, tj;
            tile_of<LOWER>(t, tiles_n, ti, tj);
            for (int kc = 0; kc < nk; ++kc, ++it) {
                const int s = (int)(it % STAGES);
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1u)) {
                    *abort_flag = 1;
                    break;
                }
                unsigned char* sa = base + s * STAGE_BYTES;
                mbar_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(sa, &ma, kc * BKC, ra0 + (int)(ti * BM), &full[s]);
                tma_load_2d(sa + OP_BYTES, &mb, kc * BKC, rb0 + (int)(tj * BN), &full[s]);
                tma_load_2d(sa + 2 * OP_BYTES, &ma_lo, kc * BKC, ra0 + (int)(ti * BM), &full[s]);
                tma_load_2d(sa + 3 * OP_BYTES, &mb_lo, kc * BKC, rb0 + (int)(tj * BN), &full[s]);
            }
        }
        if (*abort_flag) {
            // wait for this CTA's copies still in flight (the last STAGES issued)
            for (int64_t k = it - STAGES < 0 ? 0 : it - STAGES; k < it; ++k)
                mbar_wait(&full[k % STAGES], (uint32_t)(k / STAGES) & 1u);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = idesc_bf16(BM, BN);
        int64_t it = 0, tc = 0;
        for (int64_t t = blockIdx.x; t < n_tiles && !*abort_flag; t += gridDim.x, ++tc) {
            const int b = (int)(tc & 1);
            const uint32_t use = (uint32_t)(tc >> 1) & 1u;
            if (!mbar_wait(&acc_empty[b], use ^ 1u)) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dt = tmem + (uint32_t)(b * BN);
            bool ok = true;
            for (int kc = 0; kc < nk; ++kc, ++it) {
                const int s = (int)(it % STAGES);
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (*abort_flag || !mbar_wait(&full[s], ph)) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = su32(base + s * STAGE_BYTES);
                const uint64_t da = smem_desc(sa), db = smem_desc(sa + OP_BYTES);
                const uint64_t dal = smem_desc(sa + 2 * OP_BYTES), dbl = smem_desc(sa + 3 * OP_BYTES);
#pragma unroll
                for (int k = 0; k < BKC / 16; ++k) {
                    umma(dt, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (kc | k) != 0);
                    umma(dt, da + (uint64_t)(2 * k), dbl + (uint64_t)(2 * k), idesc, 1u);
                    umma(dt, dal + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, 1u);
                }
                umma_commit(&empty[s]);
            }
            if (!ok) break;
            umma_commit(&acc_full[b]);
        }
        // every product this thread issued completes before TMEM is freed
        umma_commit(drain);
        mbar_wait(drain, 0);
    } else if (warp >= 2) {
        // ---- epilogue (128 threads): C -= accumulator by TMA reduce-add of -accumulator boxes
        const int q = warp & 3;              // TMEM lane quarter this warp may access
        const int r = q * 32 + lane;         // tile row this thread drains
        const bool leader = threadIdx.x == 64;
        uint32_t chunk = 0;
        int64_t tc = 0;
        for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++tc) {
            int64_t ti, tj;
            tile_of<LOWER>(t, tiles_n, ti, tj);
            const int b = (int)(tc & 1);
            const uint32_t use = (uint32_t)(tc >> 1) & 1u;
            if (leader) {
                const bool ok = !*abort_flag && mbar_wait(&acc_full[b], use);
                if (!ok) *abort_flag = 1;
                *epi_go = ok ? 1 : 0;
            }
            named_bar(1, 128);
            if (!*epi_go) break;             // the same decision in all four warps
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += CBOX_COLS, ++chunk) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + c0), v);
                if (c0 + CBOX_COLS == BN) {   // the accumulator is in registers: hand the buffer back
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[b]);
                }
                unsigned char* box = cstage + (chunk & 1) * CBOX_BYTES;
                if (leader) bulk_wait_read<1>();   // the box used two slices ago has been read
                named_bar(1, 128);
                // row r of the box: 128 bytes, 16-byte chunk j stored at j ^ (r mod 8) (128-byte swizzle)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 o = make_float4(-__uint_as_float(v[4 * j]), -__uint_as_float(v[4 * j + 1]),
                                                 -__uint_as_float(v[4 * j + 2]), -__uint_as_float(v[4 * j + 3]));
                    *reinterpret_cast<float4*>(box + r * 128 + ((j ^ (r & 7)) << 4)) = o;
                }
                fence_proxy_async_smem();
                named_bar(1, 128);
                if (leader) {
                    tma_reduce_add_2d(&mc, cx0 + (int)(tj * BN) + c0, cy0 + (int)(ti * BM), box);
                    bulk_commit();
                }
            }
        }
        if (leader) bulk_wait_all();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) atomicExch(err, 1);
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

__global__ void k_unit_diag(float* __restrict__ X, int64_t K, int64_t ld)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < K) X[(size_t)i * ld + i] = 1.f;
}

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bool encoder()
{
    if (g_encode) return true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return true;
}

// K x K FP32, leading dimension ld (a multiple of 4): boxes of 32 x 128 with the 128-byte swizzle, the
// target of the epilogue's reduce-add
static bool make_cmap(CUtensorMap* map, float* C, int64_t K, int64_t ld)
{
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)K};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {CBOX_COLS, BM};
    cuuint32_t estr[2] = {1, 1};
    return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)C, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// rows x width BF16, row-major (width 128 or 256): boxes of 64 x 128 with the 128-byte swizzle
static bool make_map(CUtensorMap* map, const __nv_bfloat16* A, int64_t rows, int64_t width = DB)
{
    cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)width * 2};
    cuuint32_t box[2] = {BKC, BM};
    cuuint32_t estr[2] = {1, 1};
    return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)A, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace ctc

bool chol_tc_available() { return ctc::encoder(); }

cudaError_t cholesky_inverse_tc(sw_ctx* ctx, float* G, float* X, int64_t K, int64_t ld, int* d_info, int* d_err,
                                bool keep_L)
{
    using namespace ctc;
    if (K <= 0) return cudaSuccess;
    if (!encoder() || K > 0x7fff0000LL) return cudaErrorNotSupported;
    if (ld < K || (ld & 3) || ((uintptr_t)G & 15) || ((uintptr_t)X & 15)) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_diag128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DIAG_SMEM)) ||
            (e = cudaFuncSetAttribute(k_panel128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PANEL_SMEM)) ||
            (e = cudaFuncSetAttribute(k_panel_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, PT_SMEM)) ||
            (e = cudaFuncSetAttribute(k_trmm128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TRMM_SMEM)) ||
            (e = cudaFuncSetAttribute(k_tc_sub<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SUB_SMEM)) ||
            (e = cudaFuncSetAttribute(k_tc_sub<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SUB_SMEM)))
            return e;
        attr = true;
    }
    cudaStream_t st = ctx_stream(ctx);
    const bool la = ctx->opt.chol_lookahead != 0;
    if (la && !ctx->stream2) {
        if (cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ctx->stream2 = nullptr;
        }
    }
    cudaStream_t sb = la && ctx->stream2 ? ctx->stream2 : st;   // the bulk updates' stream
    const bool two = sb != st;
    // dependency events: rings of 3 for "panel k done" (P), "rest of the trailing update k done"
    // (R), "step k's bulk work done" (B) and, in 256-wide super-steps, "second panel done" (Q); no
    // dependency reaches further back than two steps
    if (two && ctx->dep_events.size() < 12) {
        while (ctx->dep_events.size() < 12) {
            cudaEvent_t ev;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return cudaErrorUnknown;
            ctx->dep_events.push_back(ev);
        }
    }
    auto evP = [&](int64_t k) { return ctx->dep_events[0 + k % 3]; };
    auto evR = [&](int64_t k) { return ctx->dep_events[3 + k % 3]; };
    auto evB = [&](int64_t k) { return ctx->dep_events[6 + k % 3]; };
    auto evQ = [&](int64_t k) { return ctx->dep_events[9 + k % 3]; };
    // scratch, double-buffered by step parity where the two streams overlap: the D blocks (128 x 128
    // FP32; two per super-step) and the panels' BF16 halves (K x W each); the inverse block rows'
    // halves (K x W each), W = 128, or 256 for two panels side by side
    const bool sup = ctx->opt.chol_super != 0;
    const int W = sup ? 2 * DB : DB;
    const int nd = sup ? 4 : 2;
    const size_t dbytes = (size_t)DB * DB * sizeof(float);
    const size_t hbytes = ((size_t)K * W * sizeof(__nv_bfloat16) + 255) & ~(size_t)255;
    // with the tensor-core panel, each D also as its swizzled BF16 split (4 boxes of 16 KB)
    const bool ptc = ctx->opt.chol_panel_tc != 0;
    const size_t swbytes = ptc ? (size_t)4 * PT_BOX : 0;
    if (ctx->ensure(&ctx->d_chol_tc, &ctx->chol_tc_cap, nd * (dbytes + swbytes) + 6 * hbytes + 256, "factor scratch") !=
        SW_OK)
        return cudaErrorMemoryAllocation;
    char* base = (char*)ctx->d_chol_tc;
    float* Dk[4] = {(float*)base, (float*)(base + dbytes), (float*)(base + 2 * dbytes), (float*)(base + 3 * dbytes)};
    uint4* Dsw[4] = {nullptr, nullptr, nullptr, nullptr};
    if (ptc)
        for (int i = 0; i < nd; ++i) Dsw[i] = (uint4*)(base + nd * dbytes + i * swbytes);
    char* hb = base + nd * (dbytes + swbytes);
    __nv_bfloat16* Ph[2] = {(__nv_bfloat16*)hb, (__nv_bfloat16*)(hb + hbytes)};
    __nv_bfloat16* Pl[2] = {(__nv_bfloat16*)(hb + 2 * hbytes), (__nv_bfloat16*)(hb + 3 * hbytes)};
    __nv_bfloat16* XTh = (__nv_bfloat16*)(hb + 4 * hbytes);
    __nv_bfloat16* XTl = (__nv_bfloat16*)(hb + 5 * hbytes);
    CUtensorMap mph[2], mpl[2], mxh, mxl, mg, mx;
    for (int b = 0; b < 2; ++b)
        if (!make_map(&mph[b], Ph[b], K, W) || !make_map(&mpl[b], Pl[b], K, W)) return cudaErrorInvalidValue;
    if (!make_map(&mxh, XTh, K, W) || !make_map(&mxl, XTl, K, W) || !make_cmap(&mg, G, K, ld) ||
        !make_cmap(&mx, X, K, ld))
        return cudaErrorInvalidValue;
    const unsigned grid_cap = (unsigned)ctx_sms(ctx);
    // the bulk updates (stream B) may leave SMs free for the next steps' chain on stream A
    const unsigned bulk_cap = (unsigned)std::max(1, ctx_sms(ctx) - (two ? ctx->opt.chol_reserve_sms : 0));
    auto tc_launch = [&](cudaStream_t s, int kid, bool lower, const CUtensorMap& a, const CUtensorMap& al,
                         const CUtensorMap& bm, const CUtensorMap& bl, const CUtensorMap& c, int cx0, int cy0,
                         int ra0, int rb0, int64_t tiles, int64_t tiles_n, double flops,
                         int depth = DB) -> cudaError_t {
        if (tiles <= 0) return cudaSuccess;
        LaunchTimer lt(ctx, kid, s);
        add_work(ctx, kid, flops);
        const unsigned g = (unsigned)std::min<int64_t>(tiles, s == st ? grid_cap : bulk_cap);
        if (lower)
            k_tc_sub<true><<<g, SUB_THREADS, SUB_SMEM, s>>>(a, al, bm, bl, c, cx0, cy0, ra0, rb0, tiles, tiles_n,
                                                           depth / BKC, d_err);
        else
            k_tc_sub<false><<<g, SUB_THREADS, SUB_SMEM, s>>>(a, al, bm, bl, c, cx0, cy0, ra0, rb0, tiles, tiles_n,
                                                            depth / BKC, d_err);
        return cudaGetLastError();
    };
    auto diag_launch = [&](int64_t j0, int bs, int slot) -> cudaError_t {
        LaunchTimer lt(ctx, K_POTRF_DIAG);
        add_work(ctx, K_POTRF_DIAG, 2.0 * (double)bs * bs * bs / 3.0);
        k_diag128<<<1, DIAG_THREADS, DIAG_SMEM, st>>>(G, ld, j0, bs, Dk[slot], d_info, keep_L ? 1 : 0, Dsw[slot]);
        return cudaGetLastError();
    };
    // the panel is launched programmatically behind its diagonal block: its row staging overlaps it
    auto panel_launch = [&](int64_t j0, int64_t r0, int64_t m, int slot, __nv_bfloat16* ph,
                            __nv_bfloat16* pl) -> cudaError_t {
        if (m <= 0) return cudaSuccess;
        LaunchTimer lt(ctx, K_TRSM_PANEL);
        add_work(ctx, K_TRSM_PANEL, (double)m * DB * DB);
        cudaLaunchConfig_t cfg = {};
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = ctx->opt.chol_pdl ? 1 : 0;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e;
        if (ptc) {
            cfg.gridDim = dim3((unsigned)((m + 127) / 128));
            cfg.blockDim = dim3(128);
            cfg.dynamicSmemBytes = PT_SMEM;
            e = cudaLaunchKernelEx(&cfg, k_panel_tc, G, ld, j0, r0, m, (const uint4*)Dsw[slot], ph, pl, W, d_err);
        } else {
            cfg.gridDim = dim3((unsigned)((m + PR - 1) / PR));
            cfg.blockDim = dim3(256);
            cfg.dynamicSmemBytes = PANEL_SMEM;
            e = cudaLaunchKernelEx(&cfg, k_panel128, G, ld, j0, r0, m, (const float*)Dk[slot], ph, pl, W);
        }
        return e ? e : cudaGetLastError();
    };
    auto trmm_launch = [&](int64_t j0, int bs, int64_t ncols, const float* D, __nv_bfloat16* xh,
                           __nv_bfloat16* xl) -> cudaError_t {
        LaunchTimer lt(ctx, K_TRINV_DIAG, sb);
        add_work(ctx, K_TRINV_DIAG, (double)bs * bs * (double)ncols);
        k_trmm128<<<(unsigned)((ncols + TC - 1) / TC), 256, TRMM_SMEM, sb>>>(X, ld, j0, bs, ncols, D, xh, xl, W);
        return cudaGetLastError();
    };
    cudaError_t e;
    // X = I
    if ((e = cudaMemsetAsync(X, 0, (size_t)K * ld * sizeof(float), st))) return e;
    {
        LaunchTimer lt(ctx, K_MISC);
        k_unit_diag<<<(unsigned)((K + 255) / 256), 256, 0, st>>>(X, K, ld);
    }
    const int64_t nb = (K + DB - 1) / DB;
    if (sup) {
        // 256-wide super-steps: blocks a = 2 s and b = 2 s + 1.  The panels of a and b sit side by side
        // in the rows of P (row g - r0a for global row g >= r0a; P_a in columns 0 .. 127, P_b in 128 ..
        // 255 from row 128 on), so the trailing matrix and the inverse's rows below b take one
        // rank-256 update per super-step: one read-modify-write pass where 128-wide steps make two.
        //   chain (stream A): diag a, panel a, block column b -= P_a P_a^T (rank 128), diag b, panel b,
        //                     block column a + 2 -= [P_a P_b][P_a P_b]^T (rank 256);
        //   bulk (stream B):  X_a <- D_a X_a, the rest of the trailing matrix (rank 256), block row b of
        //                     the inverse -= L_ba X_a (rank 128), X_b <- D_b X_b, the rows below b
        //                     -= [L_ia L_ib][X_a; X_b] (rank 256).
        // XT holds the transposed block rows side by side (X_a in columns 0 .. 127, zero in the rows of
        // block b; X_b in 128 .. 255).
        const int64_t ns = (nb + 1) / 2;
        for (int64_t si = 0; si < ns; ++si) {
            const int64_t ka = 2 * si, kbb = 2 * si + 1;
            const bool hasb = kbb < nb;
            const int64_t j0a = ka * DB;
            const int bsa = (int)(K - j0a < DB ? K - j0a : DB);
            const int64_t r0a = j0a + bsa, ma = K - r0a;
            const int64_t j0b = r0a;
            const int bsb = hasb ? (int)(K - j0b < DB ? K - j0b : DB) : 0;
            const int64_t r0b = j0b + bsb, mb = hasb ? K - r0b : 0;
            const int par = (int)(si & 1);
            const int sa = 2 * par, sbk = 2 * par + 1;
            float* Da = Dk[sa];
            float* Db = Dk[sbk];
            const int64_t Ta = (ma + BM - 1) / BM, Tb = (mb + BM - 1) / BM;
            // ---- chain
            // the buffers of parity par were last read by super-step si - 2's bulk work
            if (two && si >= 2 && (e = cudaStreamWaitEvent(st, evB(si - 2), 0))) return e;
            if ((e = diag_launch(j0a, bsa, sa))) return e;
            if ((e = panel_launch(j0a, r0a, ma, sa, Ph[par], Pl[par]))) return e;
            if (two && (e = cudaEventRecord(evP(si), st))) return e;
            if (hasb) {
                // block column b, last updated by super-step si - 1's rest
                if (two && si >= 1 && (e = cudaStreamWaitEvent(st, evR(si - 1), 0))) return e;
                if ((e = tc_launch(st, K_SYRK_TC, false, mph[par], mpl[par], mph[par], mpl[par], mg, (int)r0a, (int)r0a,
                                   0, 0, Ta, 1, 2.0 * (double)ma * std::min<int64_t>(ma, BN) * DB, DB)))
                    return e;
                if ((e = diag_launch(j0b, bsb, sbk))) return e;
                // P_b from row 128 of P, columns 128 .. 255 (mb > 0 only when block b is full)
                if ((e = panel_launch(j0b, r0b, mb, sbk, Ph[par] + (size_t)DB * W + DB, Pl[par] + (size_t)DB * W + DB)))
                    return e;
                if (two && (e = cudaEventRecord(evQ(si), st))) return e;
                if (mb > 0 &&
                    (e = tc_launch(st, K_SYRK_TC, false, mph[par], mpl[par], mph[par], mpl[par], mg, (int)r0b,
                                   (int)r0b, DB, DB, Tb, 1, 2.0 * (double)mb * std::min<int64_t>(mb, BN) * 2 * DB,
                                   2 * DB)))
                    return e;
            }
            // ---- bulk
            if (two && (e = cudaStreamWaitEvent(sb, evP(si), 0))) return e;
            if ((e = trmm_launch(j0a, bsa, r0a, Da, XTh, XTl))) return e;
            if (hasb) {
                // X_a has no entries in the columns of block b
                if ((e = cudaMemset2DAsync(XTh + (size_t)r0a * W, (size_t)W * 2, 0, (size_t)DB * 2, (size_t)bsb, sb)) ||
                    (e = cudaMemset2DAsync(XTl + (size_t)r0a * W, (size_t)W * 2, 0, (size_t)DB * 2, (size_t)bsb, sb)))
                    return e;
                if (two && (e = cudaStreamWaitEvent(sb, evQ(si), 0))) return e;
                if (Tb > 1) {
                    const int64_t T1 = Tb - 1;
                    const double mr = (double)(mb - BN);
                    if ((e = tc_launch(sb, K_SYRK_TC, true, mph[par], mpl[par], mph[par], mpl[par], mg, (int)(r0b + BN),
                                       (int)(r0b + BN), 2 * DB, 2 * DB, T1 * (T1 + 1) / 2, T1,
                                       mr * (mr + 1.0) * 2 * DB, 2 * DB)))
                        return e;
                }
            }
            if (two && (e = cudaEventRecord(evR(si), sb))) return e;
            if (hasb) {
                const int64_t Tna = (r0a + BN - 1) / BN, Tnb = (r0b + BN - 1) / BN;
                // block row b of the inverse: X_b -= L_ba X_a
                if ((e = tc_launch(sb, K_TRINV_TC, false, mph[par], mpl[par], mxh, mxl, mx, 0, (int)j0b, 0, 0, Tna, Tna,
                                   2.0 * (double)bsb * (double)r0a * DB, DB)))
                    return e;
                if ((e = trmm_launch(j0b, bsb, r0b, Db, XTh + DB, XTl + DB))) return e;
                if (mb > 0 && (e = tc_launch(sb, K_TRINV_TC, false, mph[par], mpl[par], mxh, mxl, mx, 0, (int)r0b, DB, 0,
                                             Tb * Tnb, Tnb, 2.0 * (double)mb * (double)r0b * 2 * DB, 2 * DB)))
                    return e;
            }
            if (two && (e = cudaEventRecord(evB(si), sb))) return e;
        }
        if (two && (e = cudaStreamWaitEvent(st, evB(ns - 1), 0))) return e;
        return cudaSuccess;
    }
    // Step k.  Stream A (the context's): diagonal block, panel and the trailing update's first
    // tile column (the next diagonal block's column), the chain every later step waits for.
    // Stream B: the rest of the trailing update, the inverse's block row and its update of the
    // rows below -- the bulk work, which overlaps the next steps' chain.  Without a second
    // stream everything runs in this order on A.
    for (int64_t kb = 0; kb < nb; ++kb) {
        const int64_t j0 = kb * DB;
        const int bs = (int)(K - j0 < DB ? K - j0 : DB);
        const int64_t r0 = j0 + bs, m = K - r0;
        const int par = (int)(kb & 1);
        // the buffers of parity par were last read by step kb - 2's bulk work
        if (two && kb >= 2 && (e = cudaStreamWaitEvent(st, evB(kb - 2), 0))) return e;
        {
            LaunchTimer lt(ctx, K_POTRF_DIAG);
            add_work(ctx, K_POTRF_DIAG, 2.0 * (double)bs * bs * bs / 3.0);
            k_diag128<<<1, DIAG_THREADS, DIAG_SMEM, st>>>(G, ld, j0, bs, Dk[par], d_info, keep_L ? 1 : 0, nullptr);
        }
        if ((e = cudaGetLastError())) return e;
        const int64_t T = (m + BM - 1) / BM;
        if (m > 0) {
            {
                LaunchTimer lt(ctx, K_TRSM_PANEL);
                add_work(ctx, K_TRSM_PANEL, (double)m * DB * DB);
                // launched programmatically behind the diagonal block: its row staging overlaps it
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)((m + PR - 1) / PR));
                cfg.blockDim = dim3(256);
                cfg.dynamicSmemBytes = PANEL_SMEM;
                cfg.stream = st;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                at[0].val.programmaticStreamSerializationAllowed = ctx->opt.chol_pdl ? 1 : 0;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                e = cudaLaunchKernelEx(&cfg, k_panel128, G, ld, j0, r0, m, (const float*)Dk[par], Ph[par], Pl[par], DB);
                if (e) return e;
            }
            if ((e = cudaGetLastError())) return e;
        }
        if (two && (e = cudaEventRecord(evP(kb), st))) return e;
        if (m > 0) {
            // the first tile column: column block kb + 1, last updated by step kb - 1's rest
            if (two && kb >= 1 && (e = cudaStreamWaitEvent(st, evR(kb - 1), 0))) return e;
            if ((e = tc_launch(st, K_SYRK_TC, false, mph[par], mpl[par], mph[par], mpl[par], mg, (int)r0, (int)r0, 0,
                               0, T, 1, 2.0 * (double)m * std::min<int64_t>(m, BN) * DB)))
                return e;
        }
        // ---- bulk work on stream B
        if (two && (e = cudaStreamWaitEvent(sb, evP(kb), 0))) return e;
        if (T > 1) {
            const int64_t T1 = T - 1;
            const double mr = (double)(m - BN);
            if ((e = tc_launch(sb, K_SYRK_TC, true, mph[par], mpl[par], mph[par], mpl[par], mg, (int)(r0 + BN),
                               (int)(r0 + BN), BN, BN, T1 * (T1 + 1) / 2, T1, mr * (mr + 1.0) * DB)))
                return e;
        }
        if (two && (e = cudaEventRecord(evR(kb), sb))) return e;
        {
            LaunchTimer lt(ctx, K_TRINV_DIAG, sb);
            add_work(ctx, K_TRINV_DIAG, (double)bs * bs * (double)r0);
            k_trmm128<<<(unsigned)((r0 + TC - 1) / TC), 256, TRMM_SMEM, sb>>>(X, ld, j0, bs, r0, Dk[par], XTh, XTl,
                                                                             DB);
        }
        if ((e = cudaGetLastError())) return e;
        if (m > 0) {
            const int64_t Tn = (r0 + BN - 1) / BN;
            if ((e = tc_launch(sb, K_TRINV_TC, false, mph[par], mpl[par], mxh, mxl, mx, 0, (int)r0, 0, 0, T * Tn, Tn,
                               2.0 * (double)m * (double)r0 * DB)))
                return e;
        }
        if (two && (e = cudaEventRecord(evB(kb), sb))) return e;
    }
    // the caller's stream sees the whole factorisation
    if (two && (e = cudaStreamWaitEvent(st, evB(nb - 1), 0))) return e;
    return cudaSuccess;
}

}  // namespace sw
