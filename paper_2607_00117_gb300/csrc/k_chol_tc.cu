// Cholesky factor L of the shifted passive Gram (in place, lower) and the explicit
// inverse X = L^{-1}: the preconditioner of the weight solve's reduced systems
// (Sec. 2.3).  Blocked right-looking in 128-wide steps; at step k
//
//   1. k_diag128 (one CTA): L_kk = chol(A_kk) and D_k = L_kk^{-1}.  A chain of
//      128 column steps for the factor and 128 row steps for the inverse, each
//      thread holding a fixed 4 x 8 set of the block's elements in registers
//      and one CTA barrier per step (column j, or row k of the inverse, is
//      passed through shared memory by the threads that own it);
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

// ---------------------------------------------------------------------------
// 1. Diagonal block: Cholesky and triangular inverse.  256 threads; thread
// (ty, tx) = (t / 16, t % 16) owns rows i = ty + 16 r and columns l = tx + 16 c
// (r, c < 8) of the 128 x 128 block in registers.  Cholesky in the unscaled
// form a_il -= a_ij a_lj / a_jj, two columns per CTA barrier: at a pair (j,
// j + 1) shared memory holds column j and column j + 1 as they stand before
// column j's update; every thread forms column j + 1's update and both pivots
// itself (the pivots' reciprocal square roots are the only special functions)
// and applies the rank-2 update to its elements; the owners of columns j + 2
// and j + 3 then pass them on.  The inverse X = L^{-1} runs the same way by
// pairs of rows.  The update runs unconditionally over the owned row and
// column blocks that can still change (finished rows and columns enter as
// zeros; the upper-triangle elements it also touches are never read).  The
// loops over the column block cb (factor) and the row block rb (inverse) are
// unrolled so that every register index is a compile-time constant (a
// selection by a runtime block index would put the arrays in local memory).
// ---------------------------------------------------------------------------
constexpr int DIAG_THREADS = 256;
__global__ void __launch_bounds__(DIAG_THREADS, 1) k_diag128(float* __restrict__ G, int64_t ld, int64_t j0, int bs,
                                                             float* __restrict__ D, int* info)
{
    extern __shared__ float sm[];
    float* Ls = sm;                 // DB x LP: the factor
    float* c0b = Ls + DB * LP;      // 2 x DB: column j (factor) / row k (inverse), ping-pong
    float* c1b = c0b + 2 * DB;      // 2 x DB: column j + 1 / row k + 1, before the pair's first update
    float* rdiag = c1b + 2 * DB;    // DB: 1 / L_jj
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    float a[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int i = ty + 16 * r, l = tx + 16 * c;
            a[r][c] = (i < bs && l <= i) ? G[(size_t)(j0 + i) * ld + j0 + l] : 0.f;
        }
    if (tx == 0) {
#pragma unroll
        for (int r = 0; r < 8; ++r) c0b[ty + 16 * r] = a[r][0];
    }
    if (tx == 1) {
#pragma unroll
        for (int r = 0; r < 8; ++r) c1b[ty + 16 * r] = a[r][0];
    }
    __syncthreads();
#pragma unroll
    for (int cb = 0; cb < 8; ++cb) {
#pragma unroll 1
        for (int jj = 0; jj < 16; jj += 2) {
            const int j = 16 * cb + jj, j1 = j + 1;
            if (j >= bs) break;
            const bool has1 = j1 < bs;
            const int b = (j >> 1) & 1;
            float d0 = c0b[b * DB + j];
            if (!(d0 > 0.f)) {
                if (t == 0 && info) atomicCAS(info, 0, (int)(j0 + j + 1));
                d0 = 1e-30f;
            }
            const float rs0 = rsqrtf(d0), rd0 = rs0 * rs0;
            const float cj = has1 ? c0b[b * DB + j1] : 0.f;   // a_(j+1, j)
            const float f = cj * rd0;                         // column j + 1 loses f x column j
            float d1 = has1 ? c1b[b * DB + j1] - cj * f : 1.f;
            if (!(d1 > 0.f)) {
                if (t == 0 && info) atomicCAS(info, 0, (int)(j0 + j1 + 1));
                d1 = 1e-30f;
            }
            const float rs1 = rsqrtf(d1), rd1 = rs1 * rs1;
            if (t == 0) {
                rdiag[j] = rs0;
                if (has1) rdiag[j1] = rs1;
            }
            // columns j and j + 1 are final: L_ij = a_ij / sqrt(d0), L_i(j+1) = (a_i(j+1) - f a_ij) / sqrt(d1)
            if (t < DB) {
                const float u = c0b[b * DB + t], v = c1b[b * DB + t];
                if (t >= j && t < bs) Ls[t * LP + j] = u * rs0;
                if (has1 && t >= j1 && t < bs) Ls[t * LP + j1] = (v - u * f) * rs1;
            }
            // rows and columns beyond j + 1 change; those of the blocks after cb all lie beyond it
            float p0[8], p1[8], q0[8], q1[8];
#pragma unroll
            for (int r = cb; r < 8; ++r) {
                const int i = ty + 16 * r;
                const float u = c0b[b * DB + i], v = c1b[b * DB + i];
                const bool ok = r > cb || i > j1;
                p0[r] = ok ? u * rd0 : 0.f;
                p1[r] = ok ? (v - u * f) * rd1 : 0.f;
            }
#pragma unroll
            for (int c = cb; c < 8; ++c) {
                const int l = tx + 16 * c;
                const float u = c0b[b * DB + l], v = c1b[b * DB + l];
                const bool ok = c > cb || l > j1;
                q0[c] = ok ? u : 0.f;
                q1[c] = ok ? v - u * f : 0.f;
            }
#pragma unroll
            for (int r = cb; r < 8; ++r)
#pragma unroll
                for (int c = cb; c < 8; ++c) a[r][c] -= p0[r] * q0[c] + p1[r] * q1[c];
            // the owners of columns j + 2 and j + 3 pass them on (block cb, or cb + 1 after its last pair)
            if (j + 2 < bs) {
                if (jj < 14) {
                    if (tx == jj + 2) {
#pragma unroll
                        for (int r = cb; r < 8; ++r)
                            if (ty + 16 * r > j1) c0b[(b ^ 1) * DB + ty + 16 * r] = a[r][cb];
                    }
                    if (tx == jj + 3) {
#pragma unroll
                        for (int r = cb; r < 8; ++r)
                            if (ty + 16 * r > j1) c1b[(b ^ 1) * DB + ty + 16 * r] = a[r][cb];
                    }
                } else if (cb < 7) {
                    if (tx == 0) {
#pragma unroll
                        for (int r = cb; r < 8; ++r)
                            if (ty + 16 * r > j1) c0b[(b ^ 1) * DB + ty + 16 * r] = a[r][cb < 7 ? cb + 1 : 7];
                    }
                    if (tx == 1) {
#pragma unroll
                        for (int r = cb; r < 8; ++r)
                            if (ty + 16 * r > j1) c1b[(b ^ 1) * DB + ty + 16 * r] = a[r][cb < 7 ? cb + 1 : 7];
                    }
                }
            }
            __syncthreads();
        }
    }
    // ---- inverse X = L^{-1}, right-looking by pairs of rows: with rows k and k + 1 pending
    // (every update from rows < k applied, unscaled), row k is final as x_k / L_kk, row k + 1 as
    // (x_(k+1) - L_(k+1)k row k) / L_(k+1)(k+1), and rows i > k + 1 lose L_ik row k +
    // L_i(k+1) row (k + 1).  Thread ownership as above (the factor's registers are free now).
    float (&x)[8][8] = a;
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int i = ty + 16 * r, l = tx + 16 * c;
            x[r][c] = (i == l && i < bs) ? 1.f : 0.f;
        }
    if (ty < 2) {   // rows 0 and 1 (r = 0) are pending as they are
#pragma unroll
        for (int c = 0; c < 8; ++c) (ty == 0 ? c0b : c1b)[tx + 16 * c] = x[0][c];
    }
    __syncthreads();
#pragma unroll
    for (int rb = 0; rb < 8; ++rb) {
#pragma unroll 1
        for (int kk = 0; kk < 16; kk += 2) {
            const int k = 16 * rb + kk, k1 = k + 1;
            if (k >= bs) break;
            const bool has1 = k1 < bs;
            const int b = (k >> 1) & 1;
            const float s0 = rdiag[k], s1 = has1 ? rdiag[k1] : 0.f;
            const float lkk = has1 ? Ls[k1 * LP + k] : 0.f;
            // the final rows k and k + 1 at this thread's columns (nonzero only in blocks c <= rb)
            float xk[8], xk1[8];
#pragma unroll
            for (int c = 0; c <= rb; ++c) {
                const int l = tx + 16 * c;
                xk[c] = c0b[b * DB + l] * s0;
                xk1[c] = (c1b[b * DB + l] - lkk * xk[c]) * s1;
            }
            if (ty == kk) {
#pragma unroll
                for (int c = 0; c <= rb; ++c) x[rb][c] = xk[c];
            }
            if (ty == kk + 1 && has1) {
#pragma unroll
                for (int c = 0; c <= rb; ++c) x[rb][c] = xk1[c];
            }
            float l0[8], l1[8];
#pragma unroll
            for (int r = rb; r < 8; ++r) {
                const int i = ty + 16 * r;
                const float u = Ls[i * LP + k], v = Ls[i * LP + k1];
                const bool ok = (r > rb || i > k1) && i < bs;
                l0[r] = ok ? u : 0.f;
                l1[r] = ok && has1 ? v : 0.f;
            }
#pragma unroll
            for (int r = rb; r < 8; ++r)
#pragma unroll
                for (int c = 0; c <= rb; ++c) x[r][c] -= l0[r] * xk[c] + l1[r] * xk1[c];
            // the owners of rows k + 2 and k + 3 pass them on, pending (block rb, or rb + 1)
            if (k + 2 < bs) {
                if (kk < 14) {
                    if (ty == kk + 2) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) c0b[(b ^ 1) * DB + tx + 16 * c] = x[rb][c];
                    }
                    if (ty == kk + 3) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) c1b[(b ^ 1) * DB + tx + 16 * c] = x[rb][c];
                    }
                } else if (rb < 7) {
                    if (ty == 0) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) c0b[(b ^ 1) * DB + tx + 16 * c] = x[rb < 7 ? rb + 1 : 7][c];
                    }
                    if (ty == 1) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) c1b[(b ^ 1) * DB + tx + 16 * c] = x[rb < 7 ? rb + 1 : 7][c];
                    }
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int i = ty + 16 * r, l = tx + 16 * c;
            D[i * DB + l] = (i < bs && l <= i) ? x[r][c] : 0.f;
            if (i < bs && l <= i) G[(size_t)(j0 + i) * ld + j0 + l] = Ls[i * LP + l];
        }
}

constexpr size_t DIAG_SMEM = sizeof(float) * (DB * LP + 5 * DB);

// ---------------------------------------------------------------------------
// 2. Panel: P = A D^T for m rows below the diagonal block (A = G[r0 + i][j0 ..
// j0 + 127]), in place in G, and its BF16 hi + lo halves (m x 128 row-major).
// 64 rows per CTA of 256 threads; thread (tr, tc) = (t / 16, t % 16) computes
// rows 4 tr .. 4 tr + 3 and columns 8 tc .. 8 tc + 7, reading D transposed
// (DT[l][c] = D[c][l]) so that its eight columns are two 16-byte loads.
// ---------------------------------------------------------------------------
constexpr int PR = 64;
constexpr int DTP = DB + 4;   // padded row of DT (16-byte aligned, conflict-free float4 rows)
__global__ void __launch_bounds__(256) k_panel128(float* __restrict__ G, int64_t ld, int64_t j0, int64_t r0,
                                                  int64_t m, const float* __restrict__ D,
                                                  __nv_bfloat16* __restrict__ Ph, __nv_bfloat16* __restrict__ Pl)
{
    extern __shared__ __align__(16) float sm[];
    float* As = sm;              // PR x LP
    float* DT = As + PR * LP;    // DB x DTP (16-byte aligned: PR * LP * 4 = 33 024 bytes)
    const int t = threadIdx.x;
    const int64_t row0 = (int64_t)blockIdx.x * PR;
    // many loads in flight per thread: the staging is latency-bound otherwise
#pragma unroll 8
    for (int e = t; e < PR * DB; e += 256) {
        const int i = e >> 7, l = e & (DB - 1);
        const int64_t gi = row0 + i;
        As[i * LP + l] = gi < m ? G[(size_t)(r0 + gi) * ld + j0 + l] : 0.f;
    }
#pragma unroll 4
    for (int e4 = t; e4 < DB * DB / 4; e4 += 256) {
        const float4 d4 = reinterpret_cast<const float4*>(D)[e4];
        const int c = (4 * e4) >> 7, l = (4 * e4) & (DB - 1);
        DT[l * DTP + c] = d4.x; DT[(l + 1) * DTP + c] = d4.y; DT[(l + 2) * DTP + c] = d4.z;
        DT[(l + 3) * DTP + c] = d4.w;
    }
    __syncthreads();
    const int tr = t >> 4, tc = t & 15;
    float acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;
#pragma unroll 4
    for (int l = 0; l < DB; ++l) {
        float av[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) av[r] = As[(4 * tr + r) * LP + l];
        const float4 d0 = *reinterpret_cast<const float4*>(&DT[l * DTP + 8 * tc]);
        const float4 d1 = *reinterpret_cast<const float4*>(&DT[l * DTP + 8 * tc + 4]);
        const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[r][q] += av[r] * dv[q];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t gi = row0 + 4 * tr + r;
        if (gi >= m) continue;
        float* g = G + (size_t)(r0 + gi) * ld + j0 + 8 * tc;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            g[q] = acc[r][q];
            g[q + 1] = acc[r][q + 1];
            const __nv_bfloat162 h = __floats2bfloat162_rn(acc[r][q], acc[r][q + 1]);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(acc[r][q] - __low2float(h), acc[r][q + 1] - __high2float(h));
            hw[q / 2] = (uint32_t)__bfloat16_as_ushort(h.x) | ((uint32_t)__bfloat16_as_ushort(h.y) << 16);
            lw[q / 2] = (uint32_t)__bfloat16_as_ushort(lo.x) | ((uint32_t)__bfloat16_as_ushort(lo.y) << 16);
        }
        *reinterpret_cast<uint4*>(Ph + (size_t)gi * DB + 8 * tc) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(Pl + (size_t)gi * DB + 8 * tc) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

constexpr size_t PANEL_SMEM = sizeof(float) * (PR * LP + DB * DTP);

// ---------------------------------------------------------------------------
// 4. Block row of the inverse: X[j0 + i][c] <- sum_l D[i][l] X[j0 + l][c] for
// the ncols leading columns (in place), and its transpose as BF16 hi + lo
// halves: XT[c][i] (ncols x 128 row-major).  64 columns per CTA of 256 threads;
// thread (trow, tcol) = (t / 16, t % 16) computes rows 8 trow .. 8 trow + 7 and
// columns 4 tcol .. 4 tcol + 3, reading D transposed (DT[l][i] = D[i][l]).
// ---------------------------------------------------------------------------
constexpr int TC = 64;
__global__ void __launch_bounds__(256) k_trmm128(float* __restrict__ X, int64_t ld, int64_t j0, int bs,
                                                 int64_t ncols, const float* __restrict__ D,
                                                 __nv_bfloat16* __restrict__ XTh, __nv_bfloat16* __restrict__ XTl)
{
    extern __shared__ __align__(16) float sm[];
    float* Ss = sm;                   // DB x (TC + 4)
    float* DT = Ss + DB * (TC + 4);   // DB x DTP
    __nv_bfloat16* Th = reinterpret_cast<__nv_bfloat16*>(DT + DB * DTP);   // TC x (DB + 8)
    __nv_bfloat16* Tl = Th + TC * (DB + 8);
    const int t = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * TC;
#pragma unroll 8
    for (int e = t; e < DB * TC; e += 256) {
        const int i = e / TC, cc = e % TC;
        const int64_t gc = c0 + cc;
        Ss[i * (TC + 4) + cc] = (i < bs && gc < ncols) ? X[(size_t)(j0 + i) * ld + gc] : 0.f;
    }
#pragma unroll 4
    for (int e4 = t; e4 < DB * DB / 4; e4 += 256) {
        const float4 d4 = reinterpret_cast<const float4*>(D)[e4];
        const int i = (4 * e4) >> 7, l = (4 * e4) & (DB - 1);
        DT[l * DTP + i] = d4.x; DT[(l + 1) * DTP + i] = d4.y; DT[(l + 2) * DTP + i] = d4.z;
        DT[(l + 3) * DTP + i] = d4.w;
    }
    __syncthreads();
    const int trow = t >> 4, tcol = t & 15;
    float acc[8][4];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[k][j] = 0.f;
    const int lmax = 8 * trow + 7;   // D[i][l] = 0 for l > i
#pragma unroll 4
    for (int l = 0; l <= lmax; ++l) {
        const float4 sv = *reinterpret_cast<const float4*>(&Ss[l * (TC + 4) + 4 * tcol]);
        const float4 d0 = *reinterpret_cast<const float4*>(&DT[l * DTP + 8 * trow]);
        const float4 d1 = *reinterpret_cast<const float4*>(&DT[l * DTP + 8 * trow + 4]);
        const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            acc[k][0] += dv[k] * sv.x;
            acc[k][1] += dv[k] * sv.y;
            acc[k][2] += dv[k] * sv.z;
            acc[k][3] += dv[k] * sv.w;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = 8 * trow + k;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cc = 4 * tcol + j;
            const int64_t gc = c0 + cc;
            if (i < bs && gc < ncols) X[(size_t)(j0 + i) * ld + gc] = acc[k][j];
            __nv_bfloat16 h, lo;
            split_bf16(i < bs ? acc[k][j] : 0.f, h, lo);
            Th[cc * (DB + 8) + i] = h;
            Tl[cc * (DB + 8) + i] = lo;
        }
    }
    __syncthreads();
    // coalesced rows of XT: 64 columns x 128 BF16 = 16 chunks of 16 bytes per row and half
    for (int e = t; e < TC * 16; e += 256) {
        const int cc = e >> 4, ch = e & 15;
        const int64_t gc = c0 + cc;
        if (gc >= ncols) continue;
        *reinterpret_cast<uint4*>(XTh + (size_t)gc * DB + ch * 8) =
            *reinterpret_cast<const uint4*>(Th + cc * (DB + 8) + ch * 8);
        *reinterpret_cast<uint4*>(XTl + (size_t)gc * DB + ch * 8) =
            *reinterpret_cast<const uint4*>(Tl + cc * (DB + 8) + ch * 8);
    }
}

constexpr size_t TRMM_SMEM =
    sizeof(float) * (DB * (TC + 4) + DB * DTP) + 2 * sizeof(__nv_bfloat16) * TC * (DB + 8);

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

// rows x 128 BF16, row-major (256-byte rows): boxes of 64 x 128 with the 128-byte swizzle
static bool make_map(CUtensorMap* map, const __nv_bfloat16* A, int64_t rows)
{
    cuuint64_t dims[2] = {(cuuint64_t)DB, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)DB * 2};
    cuuint32_t box[2] = {BKC, BM};
    cuuint32_t estr[2] = {1, 1};
    return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)A, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace ctc

bool chol_tc_available() { return ctc::encoder(); }

cudaError_t cholesky_inverse_tc(sw_ctx* ctx, float* G, float* X, int64_t K, int64_t ld, int* d_info, int* d_err)
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
    // (R) and "step k's bulk work done" (B); no dependency reaches further back than two steps
    if (two && ctx->dep_events.size() < 9) {
        while (ctx->dep_events.size() < 9) {
            cudaEvent_t ev;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return cudaErrorUnknown;
            ctx->dep_events.push_back(ev);
        }
    }
    auto evP = [&](int64_t k) { return ctx->dep_events[0 + k % 3]; };
    auto evR = [&](int64_t k) { return ctx->dep_events[3 + k % 3]; };
    auto evB = [&](int64_t k) { return ctx->dep_events[6 + k % 3]; };
    // scratch, double-buffered by step parity where the two streams overlap: D_k (128 x 128 FP32)
    // and the panel's BF16 halves (K x 128 each); the inverse block row's halves (K x 128 each)
    const size_t dbytes = (size_t)DB * DB * sizeof(float);
    const size_t hbytes = ((size_t)K * DB * sizeof(__nv_bfloat16) + 255) & ~(size_t)255;
    if (ctx->ensure(&ctx->d_chol_tc, &ctx->chol_tc_cap, 2 * dbytes + 6 * hbytes + 256, "factor scratch") != SW_OK)
        return cudaErrorMemoryAllocation;
    char* base = (char*)ctx->d_chol_tc;
    float* Dk[2] = {(float*)base, (float*)(base + dbytes)};
    __nv_bfloat16* Ph[2] = {(__nv_bfloat16*)(base + 2 * dbytes), (__nv_bfloat16*)(base + 2 * dbytes + hbytes)};
    __nv_bfloat16* Pl[2] = {(__nv_bfloat16*)(base + 2 * dbytes + 2 * hbytes),
                            (__nv_bfloat16*)(base + 2 * dbytes + 3 * hbytes)};
    __nv_bfloat16* XTh = (__nv_bfloat16*)(base + 2 * dbytes + 4 * hbytes);
    __nv_bfloat16* XTl = (__nv_bfloat16*)(base + 2 * dbytes + 5 * hbytes);
    CUtensorMap mph[2], mpl[2], mxh, mxl, mg, mx;
    for (int b = 0; b < 2; ++b)
        if (!make_map(&mph[b], Ph[b], K) || !make_map(&mpl[b], Pl[b], K)) return cudaErrorInvalidValue;
    if (!make_map(&mxh, XTh, K) || !make_map(&mxl, XTl, K) || !make_cmap(&mg, G, K, ld) || !make_cmap(&mx, X, K, ld))
        return cudaErrorInvalidValue;
    cudaError_t e;
    // X = I
    if ((e = cudaMemsetAsync(X, 0, (size_t)K * ld * sizeof(float), st))) return e;
    {
        LaunchTimer lt(ctx, K_MISC);
        k_unit_diag<<<(unsigned)((K + 255) / 256), 256, 0, st>>>(X, K, ld);
    }
    const unsigned grid_cap = (unsigned)ctx_sms(ctx);
    auto tc_launch = [&](cudaStream_t s, int kid, bool lower, const CUtensorMap& a, const CUtensorMap& al,
                         const CUtensorMap& bm, const CUtensorMap& bl, const CUtensorMap& c, int cx0, int cy0,
                         int ra0, int rb0, int64_t tiles, int64_t tiles_n, double flops) -> cudaError_t {
        if (tiles <= 0) return cudaSuccess;
        LaunchTimer lt(ctx, kid, s);
        add_work(ctx, kid, flops);
        const unsigned g = (unsigned)std::min<int64_t>(tiles, grid_cap);
        if (lower)
            k_tc_sub<true><<<g, SUB_THREADS, SUB_SMEM, s>>>(a, al, bm, bl, c, cx0, cy0, ra0, rb0, tiles, tiles_n,
                                                           DB / BKC, d_err);
        else
            k_tc_sub<false><<<g, SUB_THREADS, SUB_SMEM, s>>>(a, al, bm, bl, c, cx0, cy0, ra0, rb0, tiles, tiles_n,
                                                            DB / BKC, d_err);
        return cudaGetLastError();
    };
    // Step k.  Stream A (the context's): diagonal block, panel and the trailing update's first
    // tile column (the next diagonal block's column), the chain every later step waits for.
    // Stream B: the rest of the trailing update, the inverse's block row and its update of the
    // rows below -- the bulk work, which overlaps the next steps' chain.  Without a second
    // stream everything runs in this order on A.
    const int64_t nb = (K + DB - 1) / DB;
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
            k_diag128<<<1, DIAG_THREADS, DIAG_SMEM, st>>>(G, ld, j0, bs, Dk[par], d_info);
        }
        if ((e = cudaGetLastError())) return e;
        const int64_t T = (m + BM - 1) / BM;
        if (m > 0) {
            {
                LaunchTimer lt(ctx, K_TRSM_PANEL);
                add_work(ctx, K_TRSM_PANEL, (double)m * DB * DB);
                k_panel128<<<(unsigned)((m + PR - 1) / PR), 256, PANEL_SMEM, st>>>(G, ld, j0, r0, m, Dk[par],
                                                                                   Ph[par], Pl[par]);
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
            k_trmm128<<<(unsigned)((r0 + TC - 1) / TC), 256, TRMM_SMEM, sb>>>(X, ld, j0, bs, r0, Dk[par], XTh, XTl);
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
