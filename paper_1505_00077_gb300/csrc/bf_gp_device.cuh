// bf_gp_device.cuh -- sm_103a kernels of the Gauss-polynomial bilateral filter.
//
// Method: Chaudhury, "Fast and Accurate Bilateral Filtering using
// Gauss-Polynomial Decomposition", Algorithm 1 / Eqs. (7)-(11).
//
// Per plane, with h = f - t_c, R = max|h|, u = h/R, s^2 = (R/sigma_r)^2,
// E = exp(-s^2 u^2/2), channels Phi_k = E u^k (k = 0..K-1, K = N+2) and
// beta_0 = 1, beta_m = s^{2(m-1)}/m! (m >= 1), Psi_k = beta_k * S Phi_k:
//     P~ = sum_{m=1..N+1} m u^{m-1} Psi_m             (Eq. (9) / (sigma_r s))
//     Q~ = Psi_0 + s^2 u sum_{m=1..N} u^{m-1} Psi_m   (Eq. (10))
//     y  = t_c + R P~/Q~                               (Eq. (11) + Eq. (6))
// which is Eqs. (9)-(11) after substituting G_n = (s u)^n and F_n = s^n Phi_n.
// Both sums are Horner recurrences in u over descending m (3 FP32 ops per
// channel and pixel).  All channels also carry one per-plane power-of-two
// factor 2^e0 (cancels in P~/Q~) that keeps exp(-s^2 u^2/2) from underflowing
// FP32 when s^2 is large.
//
// Kernels (all FP32 arithmetic, IEEE expf and division):
//   stats_partial / stats_finalize : Algorithm 1 step 1 (mean) plus min/max;
//                                    finalize derives t_c, R, s^2, beta_k and
//                                    the scale 2^e0 (FP64).
//   row_iir / row_fir              : channel generation (steps 2-4, 7, 12) fused
//                                    with the row half of the separable filter
//                                    (steps 8, 13), scaled by beta_k, written
//                                    to the workspace [plane][k][H][Wp].
//   col_iir / col_fir              : column half of the filter fused with the
//                                    sums (steps 11, 14-16) and the division
//                                    (step 18); column-filtered planes are
//                                    never written.
//
// Recursive filter: Deriche's 4th-order Gaussian (cited in Sec. 3) written as
// h(d) = Re sum_m A_m p_m^d (two complex poles).  The line operator
// y_i = sum_j h(|i-j|) x_j (zero extension) is the sum of a causal part
// (states z_i = x_i + p z_{i-1}, output Re(A z_i)) and an anticausal part
// (states a_i = x_i + p a_{i+1}, output at i: Re(A p a_{i+1})).  A thread owns a
// chunk of C consecutive samples and runs both recursions from zero state;
// the chunk states are combined by a parallel prefix / suffix scan (the carry
// across a chunk is a multiply by p^C) and enter each output through the
// tables A p^e.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bfgp {

namespace cg = cooperative_groups;

constexpr int KMAX = 64;   // channels (order <= 62)
constexpr int NP = 2;      // complex poles of the recursive Gaussian
constexpr int CMAX = 16;   // chunk length (samples per thread)
constexpr int FIR_WMAX = 12;

// Written by stats_finalize, read by the filter kernels.
struct __align__(16) PlaneParams {
    float tc;       // centre
    float invR;     // 1 / R
    float half_s2;  // s^2 / 2
    float s2;       // s^2
    float R;        // scale
    float escale;   // 2^e0, common factor of every channel (cancels in P~/Q~)
    int mode;       // 0 = filter, 1 = copy input to output
    int pad0;
    double tc_d, R_d;
    float beta[KMAX];
};

struct __align__(16) StatPartial {
    double sum;
    float mn, mx;
    int nonfinite;
    int pad;
};

// Recursive-filter coefficients for one chunk length C (FP64 -> FP32 on the host).
struct IIRCoef {
    float pr[NP], pi[NP];                      // poles p_m
    float tr[NP][CMAX + 1], ti[NP][CMAX + 1];  // A_m p_m^e, e = 0..C  (e = 0: A_m)
    float Pr[NP][12], Pi[NP][12];              // p_m^{C 2^i}
    float wr[NP][9], wi[NP][9];                // p_m^e, e = 0..8
    float h[8];                                // h(d) = sum_m Re(A_m p_m^d), d = 0..7
    // the same numbers paired for the two-lane FMA (fma.rn.f32x2)
    float2 wc[NP][8];                          // {Re, Im} p_m^{7-i}: causal half sums
    float2 wa[NP][8];                          // {Re, Im} p_m^i: anticausal half sums
    float2 hp[15];                             // {h(|d|), h(|d+1|)}, d = -7..7 at d + 7
    float2 kc[NP][4], kcn[NP][4];              // {Re, -Im} of A_m p_m^{j+1}, A_m p_m^{j+2}, j = 0, 2, 4, 6
    float2 ka[NP][4], kan[NP][4];              // {Re, -Im} of A_m p_m^{8-j}, A_m p_m^{7-j}
};

struct FIRCoef {
    float g[FIR_WMAX + 1];  // exp(-d^2 / 2 sigma_s^2)
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ void cmadd(float &ar, float &ai, float br, float bi, float xr, float xi)
{
    // a += b * x (complex)
    ar = fmaf(br, xr, fmaf(-bi, xi, ar));
    ai = fmaf(br, xi, fmaf(bi, xr, ai));
}

__device__ __forceinline__ void cmul(float &rr, float &ri, float ar, float ai, float br, float bi)
{
    rr = fmaf(ar, br, -ai * bi);
    ri = fmaf(ar, bi, ai * br);
}

// Two FP32 FMAs in one instruction (fma.rn.f32x2, round to nearest each):
// (d.x, d.y) = (a.x b.x + c.x, a.y b.y + c.y).
__device__ __forceinline__ uint64_t pack2(float x, float y)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ void fma2(float &dx, float &dy, float ax, float ay, float bx, float by)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pack2(ax, ay)), "l"(pack2(bx, by)), "l"(pack2(dx, dy)));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(dx), "=f"(dy) : "l"(d));
}

// (rx, ry) = (ax bx, ay by), rounded to nearest
__device__ __forceinline__ void mul2(float &rx, float &ry, float ax, float ay, float bx, float by)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(ax, ay)), "l"(pack2(bx, by)));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(rx), "=f"(ry) : "l"(d));
}
// (rx, ry) = (ax bx + cx, ay by + cy)
__device__ __forceinline__ void fma2r(float &rx, float &ry, float ax, float ay, float bx, float by, float cx, float cy)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pack2(ax, ay)), "l"(pack2(bx, by)), "l"(pack2(cx, cy)));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(rx), "=f"(ry) : "l"(d));
}

// (rx, ry) = (ax - bx, ay - by), rounded to nearest
__device__ __forceinline__ void sub2(float &rx, float &ry, float ax, float ay, float bx, float by)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack2(ax, ay)), "l"(pack2(bx, by)));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(rx), "=f"(ry) : "l"(d));
}

// p^{C n} by binary powering from the table p^{C 2^i}, 0 <= n < 4096.  The
// pole index m may vary between threads: it selects, so the table stays in
// the constant bank.
__device__ __forceinline__ void cpow_tab(float &rr, float &ri, const IIRCoef &cf, int m, int n)
{
    rr = 1.f;
    ri = 0.f;
#pragma unroll
    for (int i = 0; i < 12; ++i)
        if ((n >> i) & 1) {
            const float br = m == 0 ? cf.Pr[0][i] : cf.Pr[1][i];
            const float bi = m == 0 ? cf.Pi[0][i] : cf.Pi[1][i];
            float tr, ti;
            cmul(tr, ti, rr, ri, br, bi);
            rr = tr;
            ri = ti;
        }
}

// Halves of 8 samples.  Sums over one half with zero state outside it:
//   ce[m] = sum_i p_m^{7-i} x_i   (causal state at the half's end)
//   as[m] = sum_i p_m^i x_i       (anticausal state at the half's start)
__device__ __forceinline__ void half_sums(const float *x, float (&cer)[NP], float (&cei)[NP], float (&asr)[NP],
                                          float (&asi)[NP], const IIRCoef &cf)
{
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        float a0 = x[7], a1 = 0.f, b0 = x[0], b1 = 0.f;
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            a0 = fmaf(cf.wr[m][7 - i], x[i], a0);
            a1 = fmaf(cf.wi[m][7 - i], x[i], a1);
            b0 = fmaf(cf.wr[m][i + 1], x[i + 1], b0);
            b1 = fmaf(cf.wi[m][i + 1], x[i + 1], b1);
        }
        cer[m] = a0;
        cei[m] = a1;
        asr[m] = b0;
        asi[m] = b1;
    }
}

// Response of one half to its own samples: y_j = sum_i h(|j - i|) x_i.
__device__ __forceinline__ void half_local(const float *x, float *y, const IIRCoef &cf)
{
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float v = cf.h[0] * x[j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i != j) v = fmaf(cf.h[i > j ? i - j : j - i], x[i], v);
        y[j] = v;
    }
}

// Adds the response of one half to the samples outside it, given the causal
// state c entering the half and the anticausal state a entering it from the
// right: y_j += sum_m Re(A_m p_m^{j+1} c_m) + Re(A_m p_m^{8-j} a_m).
__device__ __forceinline__ void half_correct(float *y, const float (&cr)[NP], const float (&ci)[NP],
                                             const float (&ar)[NP], const float (&ai)[NP], const IIRCoef &cf)
{
#pragma unroll
    for (int m = 0; m < NP; ++m) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float v = y[j];
            v = fmaf(cf.tr[m][j + 1], cr[m], v);
            v = fmaf(-cf.ti[m][j + 1], ci[m], v);
            v = fmaf(cf.tr[m][8 - j], ar[m], v);
            v = fmaf(-cf.ti[m][8 - j], ai[m], v);
            y[j] = v;
        }
    }
}

// half_sums, half_local and half_correct with the pairs of the coefficient
// tables in two-lane FMAs (same results: every product and sum is still one
// FP32 fused multiply-add in the same order).
__device__ __forceinline__ void half_sums2(const float *x, float (&cer)[NP], float (&cei)[NP], float (&asr)[NP],
                                           float (&asi)[NP], const IIRCoef &cf)
{
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        float a0 = x[7], a1 = 0.f, b0 = x[0], b1 = 0.f;
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            fma2(a0, a1, cf.wc[m][i].x, cf.wc[m][i].y, x[i], x[i]);
            fma2(b0, b1, cf.wa[m][i + 1].x, cf.wa[m][i + 1].y, x[i + 1], x[i + 1]);
        }
        cer[m] = a0;
        cei[m] = a1;
        asr[m] = b0;
        asi[m] = b1;
    }
}

__device__ __forceinline__ void half_local2(const float *x, float *y, const IIRCoef &cf)
{
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
        float v0, v1;
        mul2(v0, v1, cf.h[0], cf.h[0], x[j], x[j + 1]);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i == j) {
                v1 = fmaf(cf.h[1], x[i], v1);
            } else if (i == j + 1) {
                v0 = fmaf(cf.h[1], x[i], v0);
            } else {
                // pair (h(|j - i|), h(|j + 1 - i|)) = hp[j - i + 7]
                fma2(v0, v1, cf.hp[j - i + 7].x, cf.hp[j - i + 7].y, x[i], x[i]);
            }
        }
        y[j] = v0;
        y[j + 1] = v1;
    }
}

__device__ __forceinline__ void half_correct2(float *y, const float (&cr)[NP], const float (&ci)[NP],
                                              const float (&ar)[NP], const float (&ai)[NP], const IIRCoef &cf)
{
#pragma unroll
    for (int m = 0; m < NP; ++m) {
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            float v0 = y[j], v1 = y[j + 1];
            fma2(v0, v1, cf.kc[m][j >> 1].x, cf.kc[m][j >> 1].y, cr[m], cr[m]);
            fma2(v0, v1, cf.kcn[m][j >> 1].x, cf.kcn[m][j >> 1].y, ci[m], ci[m]);
            fma2(v0, v1, cf.ka[m][j >> 1].x, cf.ka[m][j >> 1].y, ar[m], ar[m]);
            fma2(v0, v1, cf.kan[m][j >> 1].x, cf.kan[m][j >> 1].y, ai[m], ai[m]);
            y[j] = v0;
            y[j + 1] = v1;
        }
    }
}

// Local recursions of one chunk from zero state.
//   y[j] = sum_m Re(A_m z_j) + Re(A_m p_m a_{j+1})   (a_C = 0)
//   e[m] = z_{C-1}   (causal state at the chunk end)
//   s[m] = a_0       (anticausal state at the chunk start)
template <int C>
__device__ __forceinline__ void chunk_local(const float (&x)[C], float (&y)[C], float (&er)[NP], float (&ei)[NP],
                                            float (&sr)[NP], float (&si)[NP], const IIRCoef &cf)
{
#pragma unroll
    for (int j = 0; j < C; ++j) y[j] = 0.f;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const float pr = cf.pr[m], pi = cf.pi[m];
        const float Ar = cf.tr[m][0], Ai = cf.ti[m][0];
        const float Br = cf.tr[m][1], Bi = cf.ti[m][1];  // A p
        float zr = 0.f, zi = 0.f;
        float ar = 0.f, ai = 0.f;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const float nzr = fmaf(pr, zr, fmaf(-pi, zi, x[j]));
            const float nzi = fmaf(pr, zi, pi * zr);
            zr = nzr;
            zi = nzi;
            y[j] = fmaf(Ar, zr, fmaf(-Ai, zi, y[j]));
            const int jj = C - 1 - j;
            y[jj] = fmaf(Br, ar, fmaf(-Bi, ai, y[jj]));
            const float nar = fmaf(pr, ar, fmaf(-pi, ai, x[jj]));
            const float nai = fmaf(pr, ai, pi * ar);
            ar = nar;
            ai = nai;
        }
        er[m] = zr;
        ei[m] = zi;
        sr[m] = ar;
        si[m] = ai;
    }
}

// y[j] += Re(A p^{j+1} cin) + Re(A p^{C-j} ain)
template <int C>
__device__ __forceinline__ void chunk_correct(float (&y)[C], const float (&cr)[NP], const float (&ci)[NP],
                                              const float (&ar)[NP], const float (&ai)[NP], const IIRCoef &cf)
{
#pragma unroll
    for (int m = 0; m < NP; ++m) {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            float v = y[j];
            v = fmaf(cf.tr[m][j + 1], cr[m], v);
            v = fmaf(-cf.ti[m][j + 1], ci[m], v);
            v = fmaf(cf.tr[m][C - j], ar[m], v);
            v = fmaf(-cf.ti[m][C - j], ai[m], v);
            y[j] = v;
        }
    }
}

// Phi_0 = E * 2^e0 with E = exp(-s^2 u^2 / 2) formed as e1 * (e1 * 2^e0),
// e1 = exp(-s^2 u^2 / 4), so neither factor leaves the FP32 range.
__device__ __forceinline__ float envelope(const PlaneParams &P, float u)
{
    const float e1 = expf(-0.5f * P.half_s2 * (u * u));
    return (e1 * P.escale) * e1;
}

// ------------------------------------------------------------------ stats

// Counters after the status word in the workspace header (byte 8 on), zeroed
// with it by the statistics pass of every call:
//   [0] pixels whose Q <= 0 (they keep their own value), [1] non-finite input values,
//   [2] planes whose exponentials leave the FP32 range, [3] bounded waits that gave up.
constexpr int NCOUNTERS = 4;
__device__ __forceinline__ unsigned long long *status_counters(uint32_t *status)
{
    return reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(status) + 8);
}
// Adds a warp's pixels with Q <= 0 to the counter and raises the flag (every lane calls).
__device__ __noinline__ void count_nonpos(uint32_t *status, int nonpos)
{
    const unsigned n = __reduce_add_sync(0xffffffffu, (unsigned)nonpos);
    if (n && (threadIdx.x & 31) == 0) {
        atomicOr(status, 0x1u);
        atomicAdd(status_counters(status), (unsigned long long)n);
    }
}


// grid (nblk, planes), block 256.  Each block reduces a band of rows.  Block
// (0, 0) also zeroes the status word of this call.
// COPY: f is host memory mapped into the device's address space (read with
// plain loads), and every value read is also stored at the same place of
// `copy` (device memory, same pitch): the input crosses the host link once,
// inside this pass.
template <bool COPY = false>
__device__ __forceinline__ void stats_partial_body(const float *__restrict__ f, int H, int W, int pitch,
                                                   int rows_per_block, int blk, StatPartial *__restrict__ out,
                                                   float *__restrict__ copy = nullptr)
{
    const int plane = 0;
    const int r0 = blk * rows_per_block;
    const int r1 = min(H, r0 + rows_per_block);
    float mn = INFINITY, mx = -INFINITY;
    double sum = 0.0;
    int bad = 0;
    const bool vec = ((pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(f) & 15) == 0);
    const float *base = f + (size_t)plane * H * pitch;
    const int nrow = r1 > r0 ? r1 - r0 : 0;
    // the band as independent (row, 4-column group) items: no load waits on another
    const int W4 = vec ? (W >> 2) : 0;
    const int items = nrow * W4;
    float acc = 0.f;
    // item i = (row r0 + r, group c4), stepped without a division per item.  Four
    // items per round, all four loads issued before any value is used, and no
    // branch on the data: the loads of a round are in flight together.
    int r = r0 + (W4 > 0 ? (int)threadIdx.x / W4 : 0), c4 = W4 > 0 ? (int)threadIdx.x % W4 : 0;
    const int dr = W4 > 0 ? (int)blockDim.x / W4 : 0, dc = W4 > 0 ? (int)blockDim.x % W4 : 0;
    for (int i = threadIdx.x; i < items; i += 4 * (int)blockDim.x) {
        float4 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool ok = i + q * (int)blockDim.x < items;
            const float4 *src = reinterpret_cast<const float4 *>(base + (size_t)r * pitch) + c4;
            v[q] = ok ? (COPY ? *src : __ldg(src)) : make_float4(NAN, NAN, NAN, NAN);
            if (COPY && ok) reinterpret_cast<float4 *>(copy + (size_t)r * pitch)[c4] = v[q];
            r += dr;
            c4 += dc;
            if (c4 >= W4) {
                c4 -= W4;
                ++r;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool ok = i + q * (int)blockDim.x < items;
            const float a[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool fin = isfinite(a[t]);
                bad += (ok && !fin) ? 1 : 0;
                acc += fin ? a[t] : 0.f;
                mn = fminf(mn, fin ? a[t] : INFINITY);
                mx = fmaxf(mx, fin ? a[t] : -INFINITY);
            }
        }
        sum += (double)acc;  // FP32 over at most 16 values, then FP64
        acc = 0.f;
    }
    sum += (double)acc;
    // the columns the 4-groups leave (all of them without vector loads)
    const int tail0 = W4 << 2, tw = W - tail0;
    const int titems = nrow * tw;
    for (int i = threadIdx.x; i < titems; i += blockDim.x) {
        const int r = r0 + i / tw, x = tail0 + (i - (i / tw) * tw);
        const float a = COPY ? base[(size_t)r * pitch + x] : __ldg(base + (size_t)r * pitch + x);
        if (COPY) copy[(size_t)r * pitch + x] = a;
        if (!isfinite(a)) {
            ++bad;
            continue;
        }
        sum += (double)a;
        mn = fminf(mn, a);
        mx = fmaxf(mx, a);
    }
    __shared__ double ssum[8];
    __shared__ float smn[8], smx[8];
    __shared__ int sbad[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
        ssum[warp] = sum;
        smn[warp] = mn;
        smx[warp] = mx;
        sbad[warp] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        StatPartial p;
        p.sum = 0.0;
        p.mn = INFINITY;
        p.mx = -INFINITY;
        p.nonfinite = 0;
        p.pad = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            p.sum += ssum[w];
            p.mn = fminf(p.mn, smn[w]);
            p.mx = fmaxf(p.mx, smx[w]);
            p.nonfinite += sbad[w];
        }
        *out = p;
    }
}

template <bool COPY>
__global__ void __launch_bounds__(256) stats_partial(const float *__restrict__ f, int H, int W, int pitch,
                                                     int rows_per_block, StatPartial *__restrict__ part,
                                                     uint32_t *__restrict__ status, float *__restrict__ copy)
{
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        *status = 0u;
        for (int i = 0; i < NCOUNTERS; ++i) status_counters(status)[i] = 0ull;
    }
    const size_t po = (size_t)blockIdx.y * H * pitch;
    stats_partial_body<COPY>(f + po, H, W, pitch, rows_per_block, blockIdx.x,
                             part + (size_t)blockIdx.y * gridDim.x + blockIdx.x, COPY ? copy + po : nullptr);
}

// 1/m, m = 0..KMAX (entry 0 unused): the beta recurrence multiplies instead of dividing.
__constant__ double c_inv[KMAX + 1] = {
    0.0, 1.0 / 1, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10, 1.0 / 11,
    1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22,
    1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29, 1.0 / 30, 1.0 / 31, 1.0 / 32, 1.0 / 33,
    1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39, 1.0 / 40, 1.0 / 41, 1.0 / 42, 1.0 / 43, 1.0 / 44,
    1.0 / 45, 1.0 / 46, 1.0 / 47, 1.0 / 48, 1.0 / 49, 1.0 / 50, 1.0 / 51, 1.0 / 52, 1.0 / 53, 1.0 / 54, 1.0 / 55,
    1.0 / 56, 1.0 / 57, 1.0 / 58, 1.0 / 59, 1.0 / 60, 1.0 / 61, 1.0 / 62, 1.0 / 63, 1.0 / 64};

// grid (planes), block 256.  Reduces one plane's partials (FP64) and writes
// its PlaneParams: t_c, R, s^2, beta_k = s^{2(k-1)}/k! (thread k, FP64
// product of s^2 / j), the common scale 2^e0 and the range flag.  ORs its
// flags into the status word (zeroed by stats_partial of the same call).
// for_backward bit 0: a constant plane is filtered (R := 1) instead of copied;
// bit 1: the joint filter's channels (beta_{2n} = beta_{2n+1} = s^{2n} / n!).
__device__ __forceinline__ void stats_finalize_body(const StatPartial *__restrict__ part, int nblk, long long npix,
                                                    int centre_given, double tc_given, double sigma_r,
                                                    double sigma_s, int K, int for_backward, int c,
                                                    PlaneParams *__restrict__ pp, uint32_t *__restrict__ status)
{
    double sum = 0.0;
    float mn = INFINITY, mx = -INFINITY;
    int bad = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        const StatPartial p = part[b];  // this plane's partials
        sum += p.sum;
        mn = fminf(mn, p.mn);
        mx = fmaxf(mx, p.mx);
        bad += p.nonfinite;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    __shared__ double ssum[8];
    __shared__ float smn[8], smx[8];
    __shared__ int sbad[8];
    __shared__ double sh_tc, sh_R, sh_s2;
    __shared__ int sh_mode;
    __shared__ float stop[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        ssum[warp] = sum;
        smn[warp] = mn;
        smx[warp] = mx;
        sbad[warp] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0;
        float MN = INFINITY, MX = -INFINITY;
        long long BAD = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            S += ssum[w];
            MN = fminf(MN, smn[w]);
            MX = fmaxf(MX, smx[w]);
            BAD += sbad[w];
        }
        const double tc = centre_given ? tc_given : S / (double)npix;
        double R = fmax((double)MX - tc, tc - (double)MN);
        int mode = BAD > 0 ? 2 : 0;  // 2: non-finite input (copy + flag)
        if (BAD > 0) atomicAdd(status_counters(status) + 1, (unsigned long long)BAD);
        if (!(R > 0.0)) {
            // constant plane: the forward copies it; for training the filter runs
            // with R = 1 (the result is independent of R), which gives y = t_c = f
            // exactly and a defined derivative
            if (!(for_backward & 1)) mode = mode ? mode : 1;
            R = 1.0;
        }
        sh_tc = tc;
        sh_R = R;
        sh_s2 = isinf(sigma_r) ? 0.0 : (R / sigma_r) * (R / sigma_r);
        sh_mode = mode;
    }
    __syncthreads();
    const double s2 = sh_s2;
    // beta_k and the log2 magnitude of the largest value of channel k, beta_k max_u E u^k
    const int k = threadIdx.x;
    double beta = 0.0;
    float lmax = -INFINITY;
    // joint filter: channels 2n and 2n + 1 carry u^n with beta = s^{2n} / n!
    const bool joint = (for_backward & 2) != 0;
    if (k < K) {
        beta = 1.0;
        const int n = joint ? (k >> 1) : k;  // power of u in the channel
        if (joint) {
            for (int j = 1; j <= n; ++j) beta *= s2 * c_inv[j];
        } else {
            for (int j = 2; j <= k; ++j) beta *= s2 * c_inv[j];
        }
        if (n >= 1 && beta > 0.0) {
            const float s2f = (float)s2;
            const float u2 = fminf(1.f, (float)n / s2f);
            lmax = log2f((float)beta) - 0.7213475f * s2f * u2 + 0.5f * (float)n * log2f(u2);
        } else {
            lmax = 0.f;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) lmax = fmaxf(lmax, __shfl_down_sync(0xffffffffu, lmax, o));
    if (lane == 0) stop[warp] = lmax;
    if (k < KMAX) pp[c].beta[k] = (k < K) ? (float)beta : 0.f;
    __syncthreads();
    if (threadIdx.x == 0) {
        float top = stop[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) top = fmaxf(top, stop[w]);
        const float s2f = (float)s2;
        const float e0 = fmaxf(0.f, ceilf(0.7213475f * s2f - 120.f));  // E 2^e0 >= 2^-120 at |u| = 1
        const float gain = 2.f * log2f(2.6f * (float)sigma_s + 2.f);
        uint32_t flags = sh_mode == 2 ? 0x2u : 0u;
        if (sh_mode == 0 && (0.3606738f * s2f > 120.f || e0 + top + gain + 2.f * log2f((float)K) > 124.f))
            flags |= 0x4u;
        PlaneParams &q = pp[c];
        q.tc = (float)sh_tc;
        q.invR = (float)(1.0 / sh_R);
        q.half_s2 = (float)(0.5 * s2);
        q.s2 = s2f;
        q.R = (float)sh_R;
        q.escale = exp2f(e0);
        q.mode = sh_mode ? 1 : 0;
        q.pad0 = (int)flags;
        q.tc_d = sh_tc;
        q.R_d = sh_R;
        if (flags) atomicOr(status, flags);
        if (flags & 0x4u) atomicAdd(status_counters(status) + 2, 1ull);
    }
}

__global__ void __launch_bounds__(256) stats_finalize(const StatPartial *__restrict__ part, int nblk,
                                                      long long npix, int centre_given, double tc_given,
                                                      double sigma_r, double sigma_s, int K, int for_backward,
                                                      PlaneParams *__restrict__ pp, uint32_t *__restrict__ status)
{
    stats_finalize_body(part + (size_t)blockIdx.x * nblk, nblk, npix, centre_given, tc_given, sigma_r, sigma_s, K,
                        for_backward, blockIdx.x, pp, status);
}

// ------------------------------------------------------------------ modes

// MODE_FWD: forward.  MODE_SAVE: forward that also writes, per pixel, the
// four sums the backward pass needs.  MODE_ADJ: backward (adjoint) pass.
// MODE_JOINT: joint (cross) filter, range weights from a guide, data from a
// second image (channels D_n = 2^e0 E u^n and U_n = D_n d, n = 0..N, with u
// and E from the guide and d = (data - t_c) / R; K = 2 (N + 1)).
enum { MODE_FWD = 0, MODE_SAVE = 1, MODE_ADJ = 2, MODE_JOINT = 3 };

// Saved per pixel by MODE_SAVE, layout [planes][4][H][W]:
//   0: P~   1: Q~   2: dp = sum_{m>=2} m (m-1) u^{m-2} Psi_m  (= dP~/du)
//   3: dq = sum_{1<=m<=N} m u^{m-1} Psi_m  (dQ~/du = s^2 dq)
// Backward accumulators per plane (FP64, in the workspace): [0] sum of dL/dy,
// [1] sum of dL/dh, [2] dL/d(s^2); zeroed by the adjoint row pass.
constexpr int NACC = 4;

struct RowArgs {
    const float *f;
    const float *gy;     // MODE_ADJ: dL/dy, same layout as f
    const float *fd;     // MODE_JOINT: the data image, same layout as f (f is the guide)
    const float *saved;  // MODE_ADJ: the MODE_SAVE sums
    float *ws;           // [planes][K][H][Wp]
    const PlaneParams *pp;
    double *acc;         // MODE_ADJ: [planes][NACC]
    int H, W, pitch, Wp, K, T, N;  // T: threads per row (power of two, 8..512)
};

__device__ __forceinline__ size_t saved_idx(int plane, int which, int H, int W, int r, int x)
{
    return (((size_t)plane * 4 + which) * H + r) * W + x;
}

__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void bar_sync_named(int id, int n)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive_named(int id, int n)
{
    asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void cluster_arrive_release()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Channel generator of the row pass for one chunk.
//   forward: Phi_k = 2^e0 E u^k (k = 0..K-1), E = exp(-s^2 u^2/2)
//   adjoint: with alpha = dL/dy R / Q~ and rho = P~ / Q~ at the pixel,
//            lambda_0 = -alpha rho,  lambda_m = alpha u^{m-1} (m - rho s^2 u) (1 <= m <= N),
//            lambda_{N+1} = alpha (N+1) u^N
//   (the adjoint of Psi_m in P~ = sum m u^{m-1} Psi_m and Q~ = Psi_0 + s^2 u sum u^{m-1} Psi_m)
template <int C, int MODE>
struct RowGen {
    // forward: v = current channel.  adjoint: v = alpha u^{m-1}; t = rho until
    // channel 0 has been formed, rho s^2 u afterwards.
    float u[C], v[C], t[C];
    float s2;
    __device__ __forceinline__ void init(const RowArgs &a, int plane, int row, bool rv, int x0, const PlaneParams &P)
    {
        s2 = P.s2;
        const float *frow = a.f + ((size_t)plane * a.H + (rv ? row : 0)) * a.pitch;
        float fv[C];
        const bool vec = ((a.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.f) & 15) == 0) && (x0 + C <= a.W);
        if (rv && vec) {
#pragma unroll
            for (int j = 0; j < C; j += 4) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(frow + x0 + j));
                fv[j] = q.x;
                fv[j + 1] = q.y;
                fv[j + 2] = q.z;
                fv[j + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) fv[j] = (rv && x0 + j < a.W) ? __ldg(frow + x0 + j) : P.tc;
        }
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const bool in = rv && (x0 + j < a.W);
            const float uu = (fv[j] - P.tc) * P.invR;
            u[j] = in ? uu : 0.f;
            if (MODE == MODE_JOINT) {
                v[j] = in ? envelope(P, uu) : 0.f;
                t[j] = in ? (__ldg(a.fd + ((size_t)plane * a.H + row) * a.pitch + x0 + j) - P.tc) * P.invR : 0.f;
            } else if (MODE != MODE_ADJ) {
                v[j] = in ? envelope(P, uu) : 0.f;
                t[j] = 0.f;
            } else {
                float al = 0.f, rho = 0.f;
                if (in) {
                    const float g = __ldg(a.gy + ((size_t)plane * a.H + row) * a.pitch + x0 + j);
                    const float Pt = __ldg(a.saved + saved_idx(plane, 0, a.H, a.W, row, x0 + j));
                    const float Qt = __ldg(a.saved + saved_idx(plane, 1, a.H, a.W, row, x0 + j));
                    if (Qt > 0.f && isfinite(g)) {
                        al = __fdiv_rn(g * P.R, Qt);
                        rho = __fdiv_rn(Pt, Qt);
                    }
                }
                v[j] = al;
                t[j] = rho;
            }
        }
    }
    // channel k into x (k increasing from 0)
    __device__ __forceinline__ void channel(int k, int N, float (&x)[C])
    {
        if (MODE == MODE_JOINT) {  // k = 2n: D_n, k = 2n + 1: U_n
            if (k & 1) {
#pragma unroll
                for (int j = 0; j < C; ++j) x[j] = v[j] * t[j];
            } else {
                if (k > 0) {
#pragma unroll
                    for (int j = 0; j < C; ++j) v[j] *= u[j];
                }
#pragma unroll
                for (int j = 0; j < C; ++j) x[j] = v[j];
            }
            return;
        }
        if (MODE != MODE_ADJ) {
            if (k > 0) {
#pragma unroll
                for (int j = 0; j < C; j += 2) mul2(v[j], v[j + 1], v[j], v[j + 1], u[j], u[j + 1]);
            }
#pragma unroll
            for (int j = 0; j < C; ++j) x[j] = v[j];
            return;
        }
        if (k == 0) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                x[j] = -v[j] * t[j];      // lambda_0 = -alpha rho
                t[j] = t[j] * s2 * u[j];  // rho s^2 u from here on
            }
            return;
        }
        const float mk = (float)k;
        if (k <= N) {
#pragma unroll
            for (int j = 0; j < C; ++j) x[j] = v[j] * (mk - t[j]);
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) x[j] = v[j] * mk;
        }
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] *= u[j];
    }
};

template <int C>
__device__ __forceinline__ void store_row_chunk(const RowArgs &a, int plane, int k, int row, bool rv, int x0,
                                                const float (&y)[C], float beta)
{
    if (!rv) return;
    float *out = a.ws + (((size_t)plane * a.K + k) * a.H + row) * a.Wp;
    if (x0 + C <= a.Wp) {
#pragma unroll
        for (int j = 0; j < C; j += 4) {
            float4 o;
            mul2(o.x, o.y, y[j], y[j + 1], beta, beta);
            mul2(o.z, o.w, y[j + 2], y[j + 3], beta, beta);
            *reinterpret_cast<float4 *>(out + x0 + j) = o;
        }
    } else {
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (x0 + j < a.Wp) out[x0 + j] = y[j] * beta;
    }
}

__device__ __forceinline__ void zero_acc(const RowArgs &a, int plane)
{
    if (threadIdx.x < NACC) a.acc[plane * NACC + threadIdx.x] = 0.0;
}

// grid (ceil(H / rows_per_cta), planes); block = max(T, 256) threads.
// Thread t of a row owns samples [t*C, (t+1)*C), two halves of 8.  Per
// channel: half sums -> chunk sums; carries by Kogge-Stone inside each warp
// (shuffles); warp totals to shared memory, in-half responses (8 x 8
// Toeplitz), one barrier; then every warp forms the carries entering it as a
// weighted sum of the other warps' totals (lane = direction x pole x source
// warp, butterfly over the source warps).
template <int C, int MODE>
__device__ __forceinline__ void row_iir_body(const RowArgs &a, const IIRCoef &cf, int grp, int plane)
{
    static_assert(C == 16, "row chunks are two halves of 8 samples");
    // warp totals [channel parity][warp slot][pole] (causal re, im, anticausal re, im); a slot is
    // rewritten two channels later, after every thread has passed the next channel's barrier
    __shared__ float4 wt[2][16][NP];
    const int T = a.T;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x;
    const int rows_per_cta = nthr / T;
    const int r_local = tid / T;
    const int t = tid % T;
    const int row = grp * rows_per_cta + r_local;
    const bool rv = row < a.H;
    const PlaneParams &P = a.pp[plane];
    const int L = T < 32 ? T : 32;  // segment width inside a warp
    const int ls = lane & (L - 1);
    const int wpr = T >> 5;         // warps per row (0 if T < 32)
    const int x0 = t * C;
    if (MODE == MODE_ADJ && grp == 0) zero_acc(a, plane);
    if (P.mode != 0) return;  // copy mode: the column pass copies f (or dL/dy)

    RowGen<C, MODE> gen;
    gen.init(a, plane, row, rv, x0, P);

    // p^{C ls} and p^{C (31 - ls)}: carry of the previous / next warps through this warp's chunks
    float qcr[NP], qci[NP], qar[NP], qai[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        cpow_tab(qcr[m], qci[m], cf, m, ls);
        cpow_tab(qar[m], qai[m], cf, m, 31 - ls);
    }

    // The carry entering warp wr of a row in direction dir, pole m, is
    // sum_w p^{512 d_w} T_w over the totals T_w of the warps before it in
    // scan order, d_w = wr - 1 - w (causal) or w - wr - 1 (anticausal).  Lane
    // (dir, m, gw) takes the terms of warps gw and gw + 8 (weight 0 where w
    // does not precede wr).
    const int wr = wpr > 0 ? warp % wpr : 0, w0 = warp - wr;
    const int gw = lane & 7, gm = (lane >> 3) & 1, gdir = lane >> 4;
    float Q0r = 0.f, Q0i = 0.f, Q1r = 0.f, Q1i = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int w = gw + 8 * h;
        const int d = gdir == 0 ? wr - 1 - w : w - wr - 1;
        if (w < wpr && d >= 0) {
            float qr, qi;
            cpow_tab(qr, qi, cf, gm, 32 * d);
            if (h == 0) {
                Q0r = qr;
                Q0i = qi;
            } else {
                Q1r = qr;
                Q1i = qi;
            }
        }
    }

#pragma unroll 1
    for (int k = 0; k < a.K; ++k) {
        float x[C];
        gen.channel(k, a.N, x);
        float hAr[NP], hAi[NP], sAr[NP], sAi[NP], hBr[NP], hBi[NP], sBr[NP], sBi[NP];
        half_sums2(x, hAr, hAi, sAr, sAi, cf);
        half_sums2(x + 8, hBr, hBi, sBr, sBi, cf);
        float er[NP], ei[NP], sr[NP], si[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            er[m] = hBr[m];
            ei[m] = hBi[m];
            cmadd(er[m], ei[m], cf.wr[m][8], cf.wi[m][8], hAr[m], hAi[m]);
            sr[m] = sAr[m];
            si[m] = sAi[m];
            cmadd(sr[m], si[m], cf.wr[m][8], cf.wi[m][8], sBr[m], sBi[m]);
        }

#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const int d = 1 << i;
            if (d >= L) break;
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const float ur = __shfl_up_sync(0xffffffffu, er[m], d);
                const float ui = __shfl_up_sync(0xffffffffu, ei[m], d);
                const float vr = __shfl_down_sync(0xffffffffu, sr[m], d);
                const float vi = __shfl_down_sync(0xffffffffu, si[m], d);
                if (ls >= d) cmadd(er[m], ei[m], cf.Pr[m][i], cf.Pi[m][i], ur, ui);
                if (ls + d < L) cmadd(sr[m], si[m], cf.Pr[m][i], cf.Pi[m][i], vr, vi);
            }
        }
        float cr[NP], ci[NP], ar[NP], ai[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float ur = __shfl_up_sync(0xffffffffu, er[m], 1);
            const float ui = __shfl_up_sync(0xffffffffu, ei[m], 1);
            const float vr = __shfl_down_sync(0xffffffffu, sr[m], 1);
            const float vi = __shfl_down_sync(0xffffffffu, si[m], 1);
            cr[m] = ls > 0 ? ur : 0.f;
            ci[m] = ls > 0 ? ui : 0.f;
            ar[m] = ls < L - 1 ? vr : 0.f;
            ai[m] = ls < L - 1 ? vi : 0.f;
        }
        float y[C];
        if (wpr > 1) {
            const int par = k & 1;
            if (lane == 31) {
#pragma unroll
                for (int m = 0; m < NP; ++m) {
                    wt[par][warp][m].x = er[m];
                    wt[par][warp][m].y = ei[m];
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int m = 0; m < NP; ++m) {
                    wt[par][warp][m].z = sr[m];
                    wt[par][warp][m].w = si[m];
                }
            }
            half_local2(x, y, cf);
            half_local2(x + 8, y + 8, cf);
            __syncthreads();  // every warp total of this channel written
            float Cr, Ci;
            {
                // source warps gw >= wpr read the row's last total (written, finite) with weight 0
                const float4 t0 = wt[par][w0 + min(gw, wpr - 1)][gm];
                cmul(Cr, Ci, Q0r, Q0i, gdir == 0 ? t0.x : t0.z, gdir == 0 ? t0.y : t0.w);
            }
            if (wpr > 8) {
                const float4 t1 = wt[par][w0 + gw + 8][gm];
                cmadd(Cr, Ci, Q1r, Q1i, gdir == 0 ? t1.x : t1.z, gdir == 0 ? t1.y : t1.w);
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                Cr += __shfl_xor_sync(0xffffffffu, Cr, o);
                Ci += __shfl_xor_sync(0xffffffffu, Ci, o);
            }
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const float cwr = __shfl_sync(0xffffffffu, Cr, (0 * 2 + m) * 8);
                const float cwi = __shfl_sync(0xffffffffu, Ci, (0 * 2 + m) * 8);
                const float awr = __shfl_sync(0xffffffffu, Cr, (1 * 2 + m) * 8);
                const float awi = __shfl_sync(0xffffffffu, Ci, (1 * 2 + m) * 8);
                cmadd(cr[m], ci[m], qcr[m], qci[m], cwr, cwi);
                cmadd(ar[m], ai[m], qar[m], qai[m], awr, awi);
            }
        } else {
            half_local2(x, y, cf);
            half_local2(x + 8, y + 8, cf);
        }
        // states entering each half: B causal p^8 c + cA, A anticausal aB + p^8 a
        float cBr[NP], cBi[NP], aAr[NP], aAi[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            cBr[m] = hAr[m];
            cBi[m] = hAi[m];
            cmadd(cBr[m], cBi[m], cf.wr[m][8], cf.wi[m][8], cr[m], ci[m]);
            aAr[m] = sBr[m];
            aAi[m] = sBi[m];
            cmadd(aAr[m], aAi[m], cf.wr[m][8], cf.wi[m][8], ar[m], ai[m]);
        }
        half_correct2(y, cr, ci, aAr, aAi, cf);
        half_correct2(y + 8, cBr, cBi, ar, ai, cf);
        store_row_chunk<C>(a, plane, k, row, rv, x0, y, P.beta[k]);
    }
}

template <int C, int MODE>
__global__ void __launch_bounds__(512) row_iir(RowArgs a, IIRCoef cf)
{
    row_iir_body<C, MODE>(a, cf, blockIdx.x, blockIdx.y);
}

// FIR row pass: the row's channel is staged in shared memory with zero halos.
// grid (ceil(H / rows_per_cta), planes); block = max(T, 256) threads.
template <int C, int WH, int MODE>
__global__ void __launch_bounds__(512) row_fir(RowArgs a, FIRCoef g)
{
    extern __shared__ float srow[];  // [2][rows_per_cta][T*C + 2*WH]
    const int T = a.T;
    const int tid = threadIdx.x;
    const int plane = blockIdx.y;
    const int rows_per_cta = blockDim.x / T;
    const int r_local = tid / T;
    const int t = tid % T;
    const int row = blockIdx.x * rows_per_cta + r_local;
    const bool rv = row < a.H;
    const PlaneParams &P = a.pp[plane];
    const int x0 = t * C;
    const int span = T * C + 2 * WH;
    if (MODE == MODE_ADJ && blockIdx.x == 0) zero_acc(a, plane);
    if (P.mode != 0) return;

    RowGen<C, MODE> gen;
    gen.init(a, plane, row, rv, x0, P);
    for (int i = tid; i < 2 * rows_per_cta * 2 * WH; i += blockDim.x) {
        const int par = i / (rows_per_cta * 2 * WH);
        const int rem = i % (rows_per_cta * 2 * WH);
        const int rl = rem / (2 * WH);
        const int h = rem % (2 * WH);
        const int pos = h < WH ? h : (T * C + h);
        srow[(par * rows_per_cta + rl) * span + pos] = 0.f;
    }

#pragma unroll 1
    for (int k = 0; k < a.K; ++k) {
        float x[C];
        gen.channel(k, a.N, x);
        float *buf = srow + ((k & 1) * rows_per_cta + r_local) * span;
#pragma unroll
        for (int j = 0; j < C; ++j) buf[WH + x0 + j] = x[j];
        __syncthreads();
        float win[C + 2 * WH];
#pragma unroll
        for (int j = 0; j < C + 2 * WH; ++j) win[j] = buf[x0 + j];
        float y[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            float acc = g.g[0] * win[j + WH];
#pragma unroll
            for (int d = 1; d <= WH; ++d) acc = fmaf(g.g[d], win[j + WH - d] + win[j + WH + d], acc);
            y[j] = acc;
        }
        store_row_chunk<C>(a, plane, k, row, rv, x0, y, P.beta[k]);
    }
}

// ------------------------------------------------------------------ column pass

struct ColArgs {
    const float *ws;  // [planes][K][H][Wp]
    const float *f;
    float *y;         // forward: output image; adjoint: dL/dh (dL/df after the finish kernel)
    const float *gy;  // MODE_ADJ: dL/dy; MODE_JOINT: the data image (f is the guide)
    float *saved;     // MODE_SAVE: written; MODE_ADJ: read
    const PlaneParams *pp;
    uint32_t *status;
    double *acc;      // MODE_ADJ
    int H, W, pitch, Wp, K, N;
    int wait_limit;   // tcgen05 column pass: polls before a wait for the tensor core gives up
    int no_mma;       // tcgen05 column pass, testing only: issue no product (every wait gives up)
};

// Per-pixel combine over descending channel m for RPT pixels.
//   forward: p = sum m u^{m-1} Psi_m (P~); q = sum_{1..N} u^{m-1} Psi_m, which
//            the last channel (m = 0) turns into Q~ = Psi_0 + s^2 u q
//   save:    also dp = sum_{m>=2} m(m-1) u^{m-2} Psi_m, dq = sum_{1..N} m u^{m-1} Psi_m
//   adjoint: with c_m the filtered adjoint channel, p = A = sum m c_m u^{m-1}, q = B = sum c_m u^m
// DSMEM: dp and dq live in shared memory (sd[j * 256] and sd[(RPT + j) * 256],
// sd pointing at this thread's column of a [2 RPT][256] block), which frees
// 2 RPT registers per thread.
// USMEM (forward, RPT a multiple of 4): the centred intensities u live in shared
// memory, us pointing at this thread's column of a [RPT / 4][256] float4 block,
// read back as float4 by every step; the RPT registers they free keep the
// column pass's working set out of local memory.
template <int RPT, int MODE, bool DSMEM = false, bool USMEM = false>
struct Combine {
    static constexpr bool SAVE_REG = MODE == MODE_SAVE && !DSMEM;
    static constexpr bool USM = USMEM && MODE == MODE_FWD && (RPT % 4) == 0;
    float u[USM ? 1 : RPT], p[RPT], q[RPT], dp[SAVE_REG ? RPT : 1], dq[SAVE_REG ? RPT : 1];
    float *sd;
    float *us;
    __device__ __forceinline__ float getu(int j) const { return USM ? us[(j >> 2) * 1024 + (j & 3)] : u[USM ? 0 : j]; }
    __device__ __forceinline__ void init(float uu, int j)
    {
        if (USM)
            us[(j >> 2) * 1024 + (j & 3)] = uu;
        else
            u[USM ? 0 : j] = uu;
        p[j] = q[j] = 0.f;
        if (MODE == MODE_SAVE) {
            if (DSMEM) {
                sd[j * 256] = 0.f;
                sd[(RPT + j) * 256] = 0.f;
            } else {
                dp[j] = dq[j] = 0.f;
            }
        }
    }
    __device__ __forceinline__ float get_dp(int j) const { return DSMEM ? sd[j * 256] : dp[j]; }
    __device__ __forceinline__ float get_dq(int j) const { return DSMEM ? sd[(RPT + j) * 256] : dq[j]; }
    __device__ __forceinline__ void step(int m, int N, float s2, const float (&y)[RPT])
    {
        if (MODE == MODE_JOINT) {  // descending m: U_n (odd m) into p, D_n (even m) into q, Horner in u
            if (m & 1) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) p[j] = fmaf(u[j], p[j], y[j]);
            } else {
#pragma unroll
                for (int j = 0; j < RPT; ++j) q[j] = fmaf(u[j], q[j], y[j]);
            }
            return;
        }
        const float mk = (float)m;
        if (MODE == MODE_ADJ) {
            // A's lowest term is m = 1 (power u^0): channel 0 does not enter it
            if (m >= 1) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) p[j] = fmaf(u[j], p[j], mk * y[j]);
            }
#pragma unroll
            for (int j = 0; j < RPT; ++j) q[j] = fmaf(u[j], q[j], y[j]);
            return;
        }
        float uv[RPT];
        if constexpr (USM) {
#pragma unroll
            for (int e = 0; e < RPT / 4; ++e) {
                const float4 v = *reinterpret_cast<const float4 *>(us + e * 1024);
                uv[4 * e] = v.x;
                uv[4 * e + 1] = v.y;
                uv[4 * e + 2] = v.z;
                uv[4 * e + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < RPT; ++j) uv[j] = u[USM ? 0 : j];
        }
        if (m == 0) {
#pragma unroll
            for (int j = 0; j < RPT; ++j) q[j] = fmaf(s2 * uv[j], q[j], y[j]);  // Q~
            return;
        }
        if (MODE == MODE_FWD && (RPT & 1) == 0) {  // the same FMAs, two per instruction
#pragma unroll
            for (int j = 0; j < RPT; j += 2) {
                if (m <= N) fma2r(q[j], q[j + 1], uv[j], uv[j + 1], q[j], q[j + 1], y[j], y[j + 1]);
                float t0, t1;
                mul2(t0, t1, mk, mk, y[j], y[j + 1]);
                fma2r(p[j], p[j + 1], uv[j], uv[j + 1], p[j], p[j + 1], t0, t1);
            }
            return;
        }
        if (MODE == MODE_SAVE) {
            const float mm1 = mk * (float)(m - 1);
            if (m >= 2) {  // dp's lowest term is m = 2 (power u^0)
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    if (DSMEM)
                        sd[j * 256] = fmaf(u[j], sd[j * 256], mm1 * y[j]);
                    else
                        dp[j] = fmaf(u[j], dp[j], mm1 * y[j]);
                }
            }
            if (m <= N) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    if (DSMEM)
                        sd[(RPT + j) * 256] = fmaf(u[j], sd[(RPT + j) * 256], mk * y[j]);
                    else
                        dq[j] = fmaf(u[j], dq[j], mk * y[j]);
                }
            }
        }
        if (m <= N) {
#pragma unroll
            for (int j = 0; j < RPT; ++j) q[j] = fmaf(u[j], q[j], y[j]);
        }
#pragma unroll
        for (int j = 0; j < RPT; ++j) p[j] = fmaf(u[j], p[j], mk * y[j]);
    }
};

struct AdjSums {
    float gy, gh, s2g;
};

// Writes the result for one pixel (r, x) of the plane.
template <int RPT, int MODE, bool DSMEM, bool USMEM>
__device__ __forceinline__ void finish_pixel(const ColArgs &a, const PlaneParams &P, int plane, int r, int x,
                                             const Combine<RPT, MODE, DSMEM, USMEM> &cb, int j, int &nonpos,
                                             AdjSums &sums)
{
    const size_t pix = ((size_t)plane * a.H + r) * a.pitch + x;
    if (MODE == MODE_ADJ) {
        const float g = __ldg(a.gy + pix);
        if (P.mode != 0) {  // the forward copied this plane: dL/df = dL/dy
            a.y[pix] = g;
            sums.gy += g;
            sums.gh += g;
            return;
        }
        const float Pt = __ldg(a.saved + saved_idx(plane, 0, a.H, a.W, r, x));
        const float Qt = __ldg(a.saved + saved_idx(plane, 1, a.H, a.W, r, x));
        const float dpv = __ldg(a.saved + saved_idx(plane, 2, a.H, a.W, r, x));
        const float dqv = __ldg(a.saved + saved_idx(plane, 3, a.H, a.W, r, x));
        const float u = cb.getu(j);
        float gdir = 0.f;
        if (Qt > 0.f && isfinite(g)) {
            const float al = __fdiv_rn(g * P.R, Qt);
            const float rho = __fdiv_rn(Pt, Qt);
            gdir = al * fmaf(-rho * P.s2, dqv, dpv);
        }
        const float E = envelope(P, u);
        const float gind = E * fmaf(-P.s2 * u, cb.q[j], cb.p[j]);
        const float gu = gind + gdir;
        float gh = gu * P.invR;
        // where the forward kept the pixel's value (Q <= 0), dL/dy reaches its own input directly
        if (!(Qt > 0.f) && isfinite(g)) gh += g;
        a.y[pix] = gh;
        sums.gy += isfinite(g) ? g : 0.f;
        sums.gh += gh;
        if (P.s2 > 0.f) sums.s2g += __fdiv_rn(u, P.s2) * gdir - 0.5f * u * u * E * cb.q[j];
        return;
    }
    if (P.mode != 0) {  // copied plane: the input (for the joint filter, its data image)
        a.y[pix] = __ldg((MODE == MODE_JOINT ? a.gy : a.f) + pix);
        return;
    }
    const float Q = cb.q[j];
    float out;
    if (!(Q > 0.f)) {
        // Eq. (11) is undefined where Q <= 0: the pixel keeps its own (data) value
        ++nonpos;
        out = __ldg((MODE == MODE_JOINT ? a.gy : a.f) + pix);
    } else {
        out = fmaf(P.R, __fdiv_rn(cb.p[j], Q), P.tc);
    }
    a.y[pix] = out;
    if (MODE == MODE_SAVE) {
        a.saved[saved_idx(plane, 0, a.H, a.W, r, x)] = cb.p[j];
        a.saved[saved_idx(plane, 1, a.H, a.W, r, x)] = Q;
        a.saved[saved_idx(plane, 2, a.H, a.W, r, x)] = cb.get_dp(j);
        a.saved[saved_idx(plane, 3, a.H, a.W, r, x)] = cb.get_dq(j);
    }
}

// Block-wide sum of the adjoint partials, then one FP64 atomic per quantity.
__device__ __forceinline__ void flush_sums(const ColArgs &a, int plane, AdjSums s)
{
    __shared__ float red[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s.gy += __shfl_down_sync(0xffffffffu, s.gy, o);
        s.gh += __shfl_down_sync(0xffffffffu, s.gh, o);
        s.s2g += __shfl_down_sync(0xffffffffu, s.s2g, o);
    }
    if (lane == 0) {
        red[0][warp] = s.gy;
        red[1][warp] = s.gh;
        red[2][warp] = s.s2g;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t0 += red[0][w];
            t1 += red[1][w];
            t2 += red[2][w];
        }
        atomicAdd(a.acc + plane * NACC + 0, t0);
        atomicAdd(a.acc + plane * NACC + 1, t1);
        atomicAdd(a.acc + plane * NACC + 2, t2);
    }
}

constexpr int COL_ROWS = 512;                                    // rows per CTA in the recursive column pass
constexpr int COL_TILE_FLOATS = (COL_ROWS + COL_ROWS / 16) * 8;  // padded [row][8 cols] tile

// Shared-memory tile row r of the 8-column strip starts at (r + r/16) * 8
// floats: a gap of 8 floats after every 16 rows puts the four chunks a warp
// reads at once on disjoint banks.
__device__ __forceinline__ int tile_off(int r) { return (r + (r >> 4)) << 3; }

__device__ __forceinline__ void cp_async16(float *dst, const float *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

constexpr int COL_TILE_BUFS = 4;  // channel tiles in flight in the recursive column pass
constexpr int COL_U_FLOATS = 16 * 256;  // the forward column pass's u (16 rows x 256 threads) after the tiles
// CTAs of 512 rows in one column cluster of the recursive column pass (more
// than 8 is a non-portable cluster size the launch has to opt into)
constexpr int COL_MAX_CTAS = 16;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Column pass for the recursive filter.  A cluster of CL CTAs covers the
// full height of an 8-column strip; CTA rank r owns rows [r*512, (r+1)*512).
// Thread (warp w, lane l): column l%8 of the strip, chunk 4w + l/8 of 16
// rows, split in two halves of 8.  Per channel (descending k):
//   1. the channel's tile (staged by cp.async two channels ahead, four
//      buffers) -> half sums -> chunk sums; carries between the 4 chunks of
//      a column in the warp by shuffles; warp totals to shared memory;
//   2. warp 0 (named barrier) turns the 8 warp totals of each column into the
//      carry entering each warp and the CTA total, and stores the CTA total
//      into the shared memory of the CTAs it enters (DSMEM);
//   3. split cluster barrier: the in-half responses (8 x 8 Toeplitz) are
//      computed while the barrier completes;
//   4. every warp adds the carry from the other CTAs (local shared memory, one
//      lane per column x pole x direction), then each half gets its entering
//      states, the out-of-half response and the Horner step.
// grid (strips * CL, planes), block 256, cluster (CL, 1, 1), CL <= MAXCTA
// (8: the portable cluster size; COL_MAX_CTAS: columns of up to 8192 rows).
// The CTAs of a cluster that share one column strip: `size` CTAs from cluster
// rank `base`, this CTA being the `rank`-th (a cluster may hold several groups,
// each on its own strip: they meet at the cluster barriers, exchange nothing).
// An inactive group has no strip: it loads and writes nothing but still meets
// every barrier.
struct ColGroup {
    int size, rank, base, active;
};

template <int C, int MODE, int MAXCTA = 8>
__device__ __forceinline__ void col_iir_body(const ColArgs &a, const IIRCoef &cf, int strip, int plane,
                                             ColGroup grp = {0, 0, 0, 1})
{
    static_assert(C == 16, "column chunks are two halves of 8 rows");
    extern __shared__ __align__(16) float tiles[];  // [COL_TILE_BUFS][COL_TILE_FLOATS]
    // [channel parity][warp][col][pole]: warp totals (causal re, im, anticausal re, im);
    // warp 0 replaces them in place by the carry entering each warp
    __shared__ float4 wt[2][8][8][NP];
    // [channel parity][source rank][col][pole][direction]: CTA totals pushed here by the other
    // CTAs of the cluster (causal ones by lower ranks, anticausal ones by higher ranks), each
    // already carried across the CTAs between source and destination; the slots no CTA writes
    // stay zero, so the carry entering this CTA is the plain sum over all slots
    __shared__ float2 inc[2][MAXCTA][8][NP][2];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int col = lane & 7, l4 = lane >> 3;
    cg::cluster_group cl = cg::this_cluster();
    // the whole cluster on one strip unless a group is given
    const int rank = grp.size ? grp.rank : (int)cl.block_rank();
    const int CL = grp.size ? grp.size : (int)cl.num_blocks();
    const int gbase = grp.size ? grp.base : 0;
    const int x = strip * 8 + col;
    const int chunk_cta = warp * 4 + l4;
    const int rbase = rank * COL_ROWS;
    const int row0 = rbase + chunk_cta * C;
    const PlaneParams &P = a.pp[plane];
    const bool filt = (P.mode == 0) && grp.active;
    const float *wsp = a.ws + (size_t)plane * a.K * a.H * a.Wp + strip * 8;

    // tile copy: 512 rows x two 16-byte halves; thread copies rows tid/2 + 128 i, i < 4
    const size_t plane_stride = (size_t)a.H * a.Wp;
    const int gr0 = rbase + (tid >> 1);
    const int src0 = gr0 * a.Wp + (tid & 1) * 4;
    const unsigned dst0 = (unsigned)__cvta_generic_to_shared(tiles + tile_off(tid >> 1) + (tid & 1) * 4);
    auto issue_tile = [&](int k) {
        const float *src = wsp + (size_t)k * plane_stride + src0;
        const unsigned dst = dst0 + (unsigned)((k & (COL_TILE_BUFS - 1)) * COL_TILE_FLOATS * sizeof(float));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool ok = filt && gr0 + 128 * i < a.H;
            // tile_off(r + 128) = tile_off(r) + 136 * 8
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst + i * 136 * 8 * 4),
                         "l"(ok ? src + (size_t)i * 128 * a.Wp : wsp), "r"(ok ? 16 : 0)
                         : "memory");
        }
    };

    // after the tiles in the dynamic shared memory: the saving forward's dp, dq; the forward's u
    Combine<C, MODE, MODE == MODE_SAVE, MODE == MODE_FWD> cb;
    cb.sd = tiles + COL_TILE_BUFS * COL_TILE_FLOATS + tid;
    cb.us = tiles + COL_TILE_BUFS * COL_TILE_FLOATS + 4 * tid;
    const float *fcol = a.f + (size_t)plane * a.H * a.pitch;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int r = row0 + j;
        const bool in = (r < a.H) && (x < a.W);
        const float fv = in ? __ldg(fcol + (size_t)r * a.pitch + x) : 0.f;
        cb.init((fv - P.tc) * P.invR, j);
    }
    // [l4][pole]: {p^{16 l4}, p^{16 (3 - l4)}} (re, im), read once per channel
    __shared__ float4 qtab[4][NP];
    if (tid < 4 * NP) {
        const int ql = tid >> 1, qm = tid & 1;
        float a0, a1, b0, b1;
        cpow_tab(a0, a1, cf, qm, ql);
        cpow_tab(b0, b1, cf, qm, 3 - ql);
        qtab[ql][qm] = make_float4(a0, a1, b0, b1);
    }
    // cross-CTA roles: lane = (dir * 2 + pole) * 8 + column
    const int gcol = lane & 7, gq = lane >> 3, gm = gq & 1, gdir = gq >> 1;
    // [warp][dir][pole]: p^{64 w}, the CTA carry crosses the warps before (causal) / after (anticausal)
    // warp w; [pole]: {p^64, p^512} for the leader's fold and pushes; read when used
    __shared__ float2 phtab[8][2][NP];
    __shared__ float4 lptab[NP];
    if (tid < 8 * 2 * NP) {
        const int pw = tid >> 2, pd = (tid >> 1) & 1, pm = tid & 1;
        float a0, a1;
        cpow_tab(a0, a1, cf, pm, 4 * (pd == 0 ? pw : 7 - pw));
        phtab[pw][pd][pm] = make_float2(a0, a1);
        if (tid < NP)
            lptab[tid] = make_float4(cf.Pr[tid][2], cf.Pi[tid][2], cf.Pr[tid][5], cf.Pi[tid][5]);
    }
    {
        float2 *z = &inc[0][0][0][0][0];
        for (int e = tid; e < 2 * MAXCTA * 8 * NP * 2; e += blockDim.x) z[e] = make_float2(0.f, 0.f);
    }
    cl.sync();  // zeroed before any peer pushes

    issue_tile(a.K - 1);
    cp_async_commit();
    if (a.K >= 2) issue_tile(a.K - 2);
    cp_async_commit();
    cp_async_wait_1();
    __syncthreads();
#pragma unroll 1
    for (int k = a.K - 1; k >= 0; --k) {
        // tile k: landed before the previous cluster barrier (or the
        // __syncthreads above); the buffer of tile k - 2 last held tile k + 2,
        // which every thread finished before arriving at that barrier
        const float *tl = tiles + (k & (COL_TILE_BUFS - 1)) * COL_TILE_FLOATS + tile_off(chunk_cta * C) + col;
        float xin[C];
#pragma unroll
        for (int j = 0; j < C; ++j) xin[j] = tl[j * 8];
        if (k >= 2) issue_tile(k - 2);
        cp_async_commit();

        float hAr[NP], hAi[NP], sAr[NP], sAi[NP], hBr[NP], hBi[NP], sBr[NP], sBi[NP];
        half_sums2(xin, hAr, hAi, sAr, sAi, cf);
        half_sums2(xin + 8, hBr, hBi, sBr, sBi, cf);
        // chunk sums: causal end state e = p^8 cA + cB, anticausal start state s = aA + p^8 aB
        float er[NP], ei[NP], sr[NP], si[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            er[m] = hBr[m];
            ei[m] = hBi[m];
            cmadd(er[m], ei[m], cf.wr[m][8], cf.wi[m][8], hAr[m], hAi[m]);
            sr[m] = sAr[m];
            si[m] = sAi[m];
            cmadd(sr[m], si[m], cf.wr[m][8], cf.wi[m][8], sBr[m], sBi[m]);
        }

        // the 4 chunks of this column inside the warp (lane stride 8)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int dd = 1 << i;
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const float ur = __shfl_up_sync(0xffffffffu, er[m], 8 * dd);
                const float ui = __shfl_up_sync(0xffffffffu, ei[m], 8 * dd);
                const float vr = __shfl_down_sync(0xffffffffu, sr[m], 8 * dd);
                const float vi = __shfl_down_sync(0xffffffffu, si[m], 8 * dd);
                if (l4 >= dd) cmadd(er[m], ei[m], cf.Pr[m][i], cf.Pi[m][i], ur, ui);
                if (l4 + dd < 4) cmadd(sr[m], si[m], cf.Pr[m][i], cf.Pi[m][i], vr, vi);
            }
        }
        float cr[NP], ci[NP], ar[NP], ai[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float ur = __shfl_up_sync(0xffffffffu, er[m], 8);
            const float ui = __shfl_up_sync(0xffffffffu, ei[m], 8);
            const float vr = __shfl_down_sync(0xffffffffu, sr[m], 8);
            const float vi = __shfl_down_sync(0xffffffffu, si[m], 8);
            cr[m] = l4 > 0 ? ur : 0.f;
            ci[m] = l4 > 0 ? ui : 0.f;
            ar[m] = l4 < 3 ? vr : 0.f;
            ai[m] = l4 < 3 ? vi : 0.f;
        }
        const int par = k & 1;
        if (l4 == 3) {
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                wt[par][warp][col][m].x = er[m];
                wt[par][warp][col][m].y = ei[m];
            }
        }
        if (l4 == 0) {
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                wt[par][warp][col][m].z = sr[m];
                wt[par][warp][col][m].w = si[m];
            }
        }
        if (warp == 0) {
            bar_sync_named(1, 256);  // all warp totals of this channel written
            float totr = 0.f, toti = 0.f;
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int w = gdir == 0 ? s : 7 - s;
                float *slot = gdir == 0 ? &wt[par][w][gcol][gm].x : &wt[par][w][gcol][gm].z;
                const float tr = slot[0], ti = slot[1];
                slot[0] = totr;
                slot[1] = toti;
                float nr, ni;
                const float4 lp = lptab[gm];
                cmul(nr, ni, lp.x, lp.y, totr, toti);
                totr = nr + tr;
                toti = ni + ti;
            }
            // push the CTA total to the CTAs it enters, later ranks (causal) or earlier ones
            // (anticausal), times p^512 per CTA crossed on the way
            float2 *own = &inc[par][rank][gcol][gm][gdir];
            const int nd = gdir == 0 ? CL - 1 - rank : rank;
            for (int d = 1; d <= nd; ++d) {
                *cl.map_shared_rank(own, gbase + (gdir == 0 ? rank + d : rank - d)) = make_float2(totr, toti);
                float nr, ni;
                const float4 lp = lptab[gm];
                cmul(nr, ni, lp.z, lp.w, totr, toti);
                totr = nr;
                toti = ni;
            }
        } else {
            bar_arrive_named(1, 256);
        }
        cp_async_wait_1();  // this thread's part of tile k - 1
        // releases the carries, the pushed CTA totals (warp 0) and tile k - 1
        cluster_arrive_release();
        float y[C];
        {
            // the tile is read again rather than kept in registers: its buffer
            // is not refilled before the next cluster barrier
            float xr[C];
#pragma unroll
            for (int j = 0; j < C; ++j) xr[j] = tl[j * 8];
            half_local2(xr, y, cf);
            half_local2(xr + 8, y + 8, cf);
        }
        cluster_wait_acquire();

        // carry entering this warp from the rest of the column: lane (dir, pole, col)
        float Wr, Wi;
        {
            const float4 w4 = wt[par][warp][gcol][gm];
            Wr = gdir == 0 ? w4.x : w4.z;
            Wi = gdir == 0 ? w4.y : w4.w;
        }
        if (CL > 1) {
            // carry from the CTAs before (causal) / after (anticausal) this one, in rank order
            const float2 *src = &inc[par][0][gcol][gm][gdir];
            float Xr = 0.f, Xi = 0.f;
#pragma unroll
            for (int s = 0; s < MAXCTA; ++s) {
                const float2 t = src[s * 8 * NP * 2];
                Xr += t.x;
                Xi += t.y;
            }
            const float2 ph = phtab[warp][gdir][gm];
            cmadd(Wr, Wi, ph.x, ph.y, Xr, Xi);
        }
        // the carries of this thread's column; states entering each half
        float cBr[NP], cBi[NP], aAr[NP], aAi[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float wcr = __shfl_sync(0xffffffffu, Wr, (0 * 2 + m) * 8 + col);
            const float wci = __shfl_sync(0xffffffffu, Wi, (0 * 2 + m) * 8 + col);
            const float war = __shfl_sync(0xffffffffu, Wr, (1 * 2 + m) * 8 + col);
            const float wai = __shfl_sync(0xffffffffu, Wi, (1 * 2 + m) * 8 + col);
            const float4 qq = qtab[l4][m];
            cmadd(cr[m], ci[m], qq.x, qq.y, wcr, wci);
            cmadd(ar[m], ai[m], qq.z, qq.w, war, wai);
            // half B: causal p^8 c + cA; half A: anticausal aB + p^8 a
            cBr[m] = hAr[m];
            cBi[m] = hAi[m];
            cmadd(cBr[m], cBi[m], cf.wr[m][8], cf.wi[m][8], cr[m], ci[m]);
            aAr[m] = sBr[m];
            aAi[m] = sBi[m];
            cmadd(aAr[m], aAi[m], cf.wr[m][8], cf.wi[m][8], ar[m], ai[m]);
        }
        half_correct2(y, cr, ci, aAr, aAi, cf);
        half_correct2(y + 8, cBr, cBi, ar, ai, cf);
        cb.step(k, a.N, P.s2, y);
    }
    // no CTA may leave while a peer can still read its shared memory
    cl.sync();
    int nonpos = 0;
    AdjSums sums = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int r = row0 + j;
        if (grp.active && r < a.H && x < a.W) finish_pixel(a, P, plane, r, x, cb, j, nonpos, sums);
    }
    if (MODE == MODE_ADJ) {
        flush_sums(a, plane, sums);
    } else {
        count_nonpos(a.status, nonpos);
    }
}

// ------------------------------------------------ tcgen05 (5th-generation tensor core) path
//
// The chunk-local work of the recursive filter on a half of 8 samples is a
// product with a fixed 16 x 8 matrix B: outputs n = 0..7 are the in-half
// responses sum_i h(|n - i|) x_i, outputs 8..15 the half's sums
// (causal end state: p_m^{7-i}; anticausal start state: p_m^i; re, im of
// poles 0 and 1).  One tcgen05.mma (kind::tf32, M = 128 halves, N = 16,
// K = 8) per 128 halves; FP32 accuracy from three TF32 products
// (A_hi B_hi + A_hi B_lo + A_lo B_hi, operands split with round-to-nearest).
// A and B sit in shared memory in the K-major core-matrix layout without
// swizzle: element (row r, k) at (r/8)*256 + (k/4)*128 + (r%8)*16 + (k%4)*4
// bytes (core matrices of 8 rows x 16 bytes; 128 bytes between the two along
// K, 256 bytes between row groups).  D (FP32) goes to tensor memory, row r in
// lane r, output n in column n, and comes back with tcgen05.ld.

struct UMat {
    float hi[128], lo[128];  // B (16 x 8) in the core-matrix layout, TF32 high part and FP32 remainder
};

constexpr uint32_t UMMA_LBO = 128, UMMA_SBO = 256;
// kind::tf32 instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t UMMA_IDESC_M128_N16 = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);


__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((UMMA_LBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((UMMA_SBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                 "l"(a), "l"(b), "r"(UMMA_IDESC_M128_N16), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Waits for the phase of parity `parity` of the mbarrier; gives up after
// `limit` polls and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit)
{
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Writes the 8 samples of one half as row r of the A operand (TF32 high parts
// to ahi, FP32 remainders to alo).
__device__ __forceinline__ void umma_put_row(float *ahi, float *alo, int r, const float *x)
{
    // Veltkamp split with 2^13 + 1: h keeps the leading 11 significant bits
    // (round to nearest), so it is exact in TF32; l = x - h is exact in FP32.
    float h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float c = __fmul_rn(x[i], 8193.f);
        h[i] = __fsub_rn(c, __fsub_rn(c, x[i]));
        l[i] = __fsub_rn(x[i], h[i]);
    }
    const int o = (r >> 3) * 64 + (r & 7) * 4;
    *reinterpret_cast<float4 *>(ahi + o) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(ahi + o + 32) = make_float4(h[4], h[5], h[6], h[7]);
    *reinterpret_cast<float4 *>(alo + o) = make_float4(l[0], l[1], l[2], l[3]);
    *reinterpret_cast<float4 *>(alo + o + 32) = make_float4(l[4], l[5], l[6], l[7]);
}

constexpr int TC5_TILE_BUFS = 3;
constexpr int TC5_SMEM_BYTES = (TC5_TILE_BUFS * COL_TILE_FLOATS + 8 * 1024 + 256) * 4;
constexpr int MBAR_LIMIT = 1 << 22;

// Column pass for the recursive filter with the half-chunk products on
// tcgen05.  Same cluster, thread and carry layout as col_iir; per channel k:
//   a. wait for the MMAs of channel k (issued one step earlier), read the
//      half sums from tensor memory;
//   b. chunk sums, carries in the warp, warp 0 -> carries per warp and CTA
//      totals pushed to the peers, cluster barrier (which also publishes
//      tile k - 1);
//   c. split tile k - 1 into the A operand and issue its MMAs (thread 0), so
//      the tensor core works while this thread finishes channel k;
//   d. carries from the other CTAs, in-half responses from tensor memory,
//      out-of-half responses, Horner step.
// Tiles are staged by cp.async two channels ahead (three buffers); D is
// double-buffered in tensor memory by channel parity (128 columns).
// Thread (warp w, lane l) owns rows 16 (4w + l/8) .. + 15 of column l % 8;
// its half s is row 32 (w % 4) + l of MMA tile 2 (w / 4) + s (tensor-memory
// columns 16 t .. 16 t + 15; a warp reads lanes 32 (w % 4) .. + 31).
template <int MODE>
__device__ __forceinline__ void col_tc5_body(const ColArgs &a, const IIRCoef &cf, const UMat &um, int strip, int plane)
{
    constexpr int C = 16;
    extern __shared__ __align__(1024) float dsm[];
    float *tiles = dsm;                                  // [3][COL_TILE_FLOATS]
    float *sA = dsm + TC5_TILE_BUFS * COL_TILE_FLOATS;   // [4 tiles][hi, lo][1024]
    float *sB = sA + 8 * 1024;                           // [hi, lo][128]
    __shared__ float4 wt[2][8][8][NP];
    __shared__ float2 inc[2][8][8][NP][2];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int col = lane & 7, l4 = lane >> 3;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int CL = (int)cl.num_blocks();
    const int x = strip * 8 + col;
    const int chunk_cta = warp * 4 + l4;
    const int rbase = rank * COL_ROWS;
    const int row0 = rbase + chunk_cta * C;
    const PlaneParams &P = a.pp[plane];
    const bool filt = (P.mode == 0);
    const float *wsp = a.ws + (size_t)plane * a.K * a.H * a.Wp + strip * 8;
    const uint32_t mb = smem_u32(&mbar);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(smem_u32(&tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    sB[tid] = tid < 128 ? um.hi[tid] : um.lo[tid - 128];

    // tile copy: 512 rows x two 16-byte halves; thread copies rows tid/2 + 128 i, i < 4
    const size_t plane_stride = (size_t)a.H * a.Wp;
    const int gr0 = rbase + (tid >> 1);
    const int src0 = gr0 * a.Wp + (tid & 1) * 4;
    const unsigned dst0 = smem_u32(tiles + tile_off(tid >> 1) + (tid & 1) * 4);
    auto issue_tile = [&](int k) {
        const float *src = wsp + (size_t)k * plane_stride + src0;
        const unsigned dst = dst0 + (unsigned)((k % TC5_TILE_BUFS) * COL_TILE_FLOATS * sizeof(float));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool ok = filt && gr0 + 128 * i < a.H;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst + i * 136 * 8 * 4),
                         "l"(ok ? src + (size_t)i * 128 * a.Wp : wsp), "r"(ok ? 16 : 0)
                         : "memory");
        }
    };
    // A rows of this thread's two halves, and the tensor-memory address of its rows
    const int arow = 32 * (warp & 3) + lane;
    const int atile = 2 * (warp >> 2);
    auto split_tile = [&](int k) {
        const float *tl = tiles + (k % TC5_TILE_BUFS) * COL_TILE_FLOATS + tile_off(chunk_cta * C) + col;
        float xv[C];
#pragma unroll
        for (int j = 0; j < C; ++j) xv[j] = tl[j * 8];
#pragma unroll
        for (int s = 0; s < 2; ++s)
            umma_put_row(sA + (atile + s) * 2048, sA + (atile + s) * 2048 + 1024, arow, xv + 8 * s);
        fence_proxy_async();
    };
    auto issue_mma = [&](uint32_t tmem) {
        const uint64_t bhi = umma_desc(smem_u32(sB)), blo = umma_desc(smem_u32(sB + 128));
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint64_t ahi = umma_desc(smem_u32(sA + t * 2048)), alo = umma_desc(smem_u32(sA + t * 2048 + 1024));
            const uint32_t d = tmem + 16 * t;
            umma_tf32(d, ahi, bhi, 0);
            umma_tf32(d, ahi, blo, 1);
            umma_tf32(d, alo, bhi, 1);
        }
        umma_commit(mb);
    };

    Combine<C, MODE> cb;
    const float *fcol = a.f + (size_t)plane * a.H * a.pitch;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int r = row0 + j;
        const bool in = (r < a.H) && (x < a.W);
        const float fv = in ? __ldg(fcol + (size_t)r * a.pitch + x) : 0.f;
        cb.init((fv - P.tc) * P.invR, j);
    }
    float qcr[NP], qci[NP], qar[NP], qai[NP];  // p^{16 l4}, p^{16 (3 - l4)}
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        cpow_tab(qcr[m], qci[m], cf, m, l4);
        cpow_tab(qar[m], qai[m], cf, m, 3 - l4);
    }
    const int gcol = lane & 7, gq = lane >> 3, gm = gq & 1, gdir = gq >> 1;
    float Phr, Phi;
    cpow_tab(Phr, Phi, cf, gm, 4 * (gdir == 0 ? warp : 7 - warp));
    const float p4r = gm == 0 ? cf.Pr[0][2] : cf.Pr[1][2], p4i = gm == 0 ? cf.Pi[0][2] : cf.Pi[1][2];
    const float p32r = gm == 0 ? cf.Pr[0][5] : cf.Pr[1][5], p32i = gm == 0 ? cf.Pi[0][5] : cf.Pi[1][5];
    const int nsteps = gdir == 0 ? rank : CL - 1 - rank;

    issue_tile(a.K - 1);
    cp_async_commit();
    if (a.K >= 2) issue_tile(a.K - 2);
    cp_async_commit();
    cp_async_wait_1();
    __syncthreads();  // tile K-1 visible
    split_tile(a.K - 1);
    tc_fence_before();
    __syncthreads();  // A of channel K-1, B, the mbarrier and the tensor-memory address visible
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 16 * atile;
    if (tid == 0 && !a.no_mma) issue_mma(tmem + 64 * ((a.K - 1) & 1));
    uint32_t phase = 0;
    // stop: a wait for the tensor core gave up (CTA-uniform).  From then on no product is
    // issued and tensor memory is not read; the CTA keeps its place in every cluster barrier
    // (its peers wait on them), and before freeing tensor memory it waits once more, again
    // bounded, for the products it gave up on.
    bool stop = false;
#pragma unroll 1
    for (int k = a.K - 1; k >= 0; --k) {
        // a. half sums of channel k
        const bool ok = stop || mbar_wait(mb, phase, a.wait_limit);
        stop = __syncthreads_or(!ok) != 0;
        const uint32_t tk = trow + 64 * (k & 1);  // D of channel k: tensor-memory columns 64 (k & 1) ..
        float d0[8], d1[8];                       // half sums of the two halves (outputs 8..15)
        if (!stop) {
            phase ^= 1u;
            tc_fence_after();
            tmem_ld8(tk + 8, d0);
            tmem_ld8(tk + 16 + 8, d1);
            tmem_wait_ld();
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) d0[j] = d1[j] = 0.f;
        }
        if (k >= 2) issue_tile(k - 2);
        cp_async_commit();

        // b. chunk sums: causal end p^8 cA + cB, anticausal start aA + p^8 aB; carries in the warp
        float er[NP], ei[NP], sr[NP], si[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            er[m] = d1[2 * m];
            ei[m] = d1[1 + 2 * m];
            cmadd(er[m], ei[m], cf.wr[m][8], cf.wi[m][8], d0[2 * m], d0[1 + 2 * m]);
            sr[m] = d0[4 + 2 * m];
            si[m] = d0[5 + 2 * m];
            cmadd(sr[m], si[m], cf.wr[m][8], cf.wi[m][8], d1[4 + 2 * m], d1[5 + 2 * m]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int dd = 1 << i;
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const float ur = __shfl_up_sync(0xffffffffu, er[m], 8 * dd);
                const float ui = __shfl_up_sync(0xffffffffu, ei[m], 8 * dd);
                const float vr = __shfl_down_sync(0xffffffffu, sr[m], 8 * dd);
                const float vi = __shfl_down_sync(0xffffffffu, si[m], 8 * dd);
                if (l4 >= dd) cmadd(er[m], ei[m], cf.Pr[m][i], cf.Pi[m][i], ur, ui);
                if (l4 + dd < 4) cmadd(sr[m], si[m], cf.Pr[m][i], cf.Pi[m][i], vr, vi);
            }
        }
        float cr[NP], ci[NP], ar[NP], ai[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float ur = __shfl_up_sync(0xffffffffu, er[m], 8);
            const float ui = __shfl_up_sync(0xffffffffu, ei[m], 8);
            const float vr = __shfl_down_sync(0xffffffffu, sr[m], 8);
            const float vi = __shfl_down_sync(0xffffffffu, si[m], 8);
            cr[m] = l4 > 0 ? ur : 0.f;
            ci[m] = l4 > 0 ? ui : 0.f;
            ar[m] = l4 < 3 ? vr : 0.f;
            ai[m] = l4 < 3 ? vi : 0.f;
        }
        const int par = k & 1;
        if (l4 == 3) {
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                wt[par][warp][col][m].x = er[m];
                wt[par][warp][col][m].y = ei[m];
            }
        }
        if (l4 == 0) {
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                wt[par][warp][col][m].z = sr[m];
                wt[par][warp][col][m].w = si[m];
            }
        }
        if (warp == 0) {
            bar_sync_named(1, 256);  // all warp totals of this channel written
            float totr = 0.f, toti = 0.f;
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int w = gdir == 0 ? s : 7 - s;
                float *slot = gdir == 0 ? &wt[par][w][gcol][gm].x : &wt[par][w][gcol][gm].z;
                const float tr = slot[0], ti = slot[1];
                slot[0] = totr;
                slot[1] = toti;
                float nr, ni;
                cmul(nr, ni, p4r, p4i, totr, toti);
                totr = nr + tr;
                toti = ni + ti;
            }
            float2 *own = &inc[par][rank][gcol][gm][gdir];
            for (int r = gdir == 0 ? rank + 1 : 0; r < (gdir == 0 ? CL : rank); ++r)
                *cl.map_shared_rank(own, r) = make_float2(totr, toti);
        } else {
            bar_arrive_named(1, 256);
        }

        cp_async_wait_1();  // this thread's part of tile k - 1
        // releases the carries, the pushed CTA totals (warp 0) and tile k - 1
        cluster_arrive_release();
        cluster_wait_acquire();

        // c. MMAs of channel k - 1, running while this thread finishes channel k
        if (k >= 1 && !stop) {
            split_tile(k - 1);
            if (warp == 0) {
                // every row of A written and fenced; D of channel k + 1 (same columns) read by every thread
                bar_sync_named(3, 256);
                if (lane == 0 && !a.no_mma) {
                    tc_fence_after();
                    issue_mma(tmem + 64 * ((k - 1) & 1));
                }
                __syncwarp();
            } else {
                bar_arrive_named(3, 256);
            }
        }

        // d. carries and the out-of-half responses
        float Wr, Wi;
        {
            const float4 w4 = wt[par][warp][gcol][gm];
            Wr = gdir == 0 ? w4.x : w4.z;
            Wi = gdir == 0 ? w4.y : w4.w;
        }
        if (CL > 1) {
            const float2 *src = gdir == 0 ? &inc[par][0][gcol][gm][0] : &inc[par][CL - 1][gcol][gm][1];
            const int step = gdir == 0 ? 8 * NP * 2 : -8 * NP * 2;
            float Xr = 0.f, Xi = 0.f;
#pragma unroll
            for (int s = 0; s < 7; ++s) {
                if (s < nsteps) {
                    const float2 t = src[s * step];
                    float nr, ni;
                    cmul(nr, ni, p32r, p32i, Xr, Xi);
                    Xr = nr + t.x;
                    Xi = ni + t.y;
                }
            }
            cmadd(Wr, Wi, Phr, Phi, Xr, Xi);
        }
        float cBr[NP], cBi[NP], aAr[NP], aAi[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float wcr = __shfl_sync(0xffffffffu, Wr, (0 * 2 + m) * 8 + col);
            const float wci = __shfl_sync(0xffffffffu, Wi, (0 * 2 + m) * 8 + col);
            const float war = __shfl_sync(0xffffffffu, Wr, (1 * 2 + m) * 8 + col);
            const float wai = __shfl_sync(0xffffffffu, Wi, (1 * 2 + m) * 8 + col);
            cmadd(cr[m], ci[m], qcr[m], qci[m], wcr, wci);
            cmadd(ar[m], ai[m], qar[m], qai[m], war, wai);
            cBr[m] = d0[2 * m];
            cBi[m] = d0[1 + 2 * m];
            cmadd(cBr[m], cBi[m], cf.wr[m][8], cf.wi[m][8], cr[m], ci[m]);
            aAr[m] = d1[4 + 2 * m];
            aAi[m] = d1[5 + 2 * m];
            cmadd(aAr[m], aAi[m], cf.wr[m][8], cf.wi[m][8], ar[m], ai[m]);
        }
        float y[C];
        {
            float l0[8], l1[8];  // in-half responses (outputs 0..7)
            if (!stop) {
                tmem_ld8(tk, l0);
                tmem_ld8(tk + 16, l1);
                tmem_wait_ld();
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) l0[j] = l1[j] = 0.f;
            }
            tc_fence_before();  // D of channel k is read before this thread reaches barrier 3 again
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                y[j] = l0[j];
                y[8 + j] = l1[j];
            }
        }
        half_correct(y, cr, ci, aAr, aAi, cf);
        half_correct(y + 8, cBr, cBi, ar, ai, cf);
        cb.step(k, a.N, P.s2, y);
    }
    // no CTA may leave while a peer can still write to or read its shared memory
    tc_fence_before();
    cl.sync();
    if (warp == 0) {
        // after a give-up the products of the channel waited for may still be running: wait for
        // them once more (bounded) before their accumulators are freed
        if (stop) (void)mbar_wait(mb, phase, a.wait_limit);
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem) : "memory");
    }
    if (stop && tid == 0) {
        atomicOr(a.status, 0x8u);
        atomicAdd(status_counters(a.status) + 3, 1ull);
    }
    int nonpos = 0;
    AdjSums sums = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int r = row0 + j;
        if (!(r < a.H && x < a.W)) continue;
        if (stop) {  // no result: the plane is written as copied (the backward: no gradient)
            const size_t pix = ((size_t)plane * a.H + r) * a.pitch + x;
            a.y[pix] = MODE == MODE_ADJ ? 0.f : __ldg((MODE == MODE_JOINT ? a.gy : a.f) + pix);
        } else {
            finish_pixel<C, MODE>(a, P, plane, r, x, cb, j, nonpos, sums);
        }
    }
    if (MODE == MODE_ADJ) {
        flush_sums(a, plane, sums);
    } else {
        count_nonpos(a.status, nonpos);
    }
}

template <int MODE>
__global__ void __launch_bounds__(256, MODE == MODE_SAVE ? 1 : 2) col_tc5(ColArgs a, IIRCoef cf, UMat um)
{
    col_tc5_body<MODE>(a, cf, um, blockIdx.x / (int)cg::this_cluster().num_blocks(), blockIdx.y);
}

template <int C, int MODE, int MAXCTA = 8>
__global__ void __launch_bounds__(256, 2) col_iir(ColArgs a, IIRCoef cf)
{
    col_iir_body<C, MODE, MAXCTA>(a, cf, blockIdx.x / (int)cg::this_cluster().num_blocks(), blockIdx.y);
}

// Column pass for the FIR filter: 2-D tiles of 32 columns x 64 rows; the
// channel's tile plus a WH-row halo is staged in shared memory.
// grid (ceil(W/32), ceil(H/64), planes), block 256 (32 columns x 8 row groups of 8).
template <int WH, int MODE>
__global__ void __launch_bounds__(256) col_fir(ColArgs a, FIRCoef g)
{
    constexpr int TH = 64, RPT = 8;
    __shared__ float tile[TH + 2 * WH][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int plane = blockIdx.z;
    const int x = blockIdx.x * 32 + tx;
    const int rbase = blockIdx.y * TH;
    const PlaneParams &P = a.pp[plane];
    const bool filt = (P.mode == 0);
    Combine<RPT, MODE> cb;
    const float *fp = a.f + (size_t)plane * a.H * a.pitch;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = rbase + ty * RPT + j;
        const bool in = (r < a.H) && (x < a.W);
        const float fv = in ? __ldg(fp + (size_t)r * a.pitch + x) : 0.f;
        cb.init((fv - P.tc) * P.invR, j);
    }
    const float *wsp = a.ws + (size_t)plane * a.K * a.H * a.Wp;
    if (filt) {
#pragma unroll 1
        for (int k = a.K - 1; k >= 0; --k) {
            const float *src = wsp + (size_t)k * a.H * a.Wp;
            __syncthreads();
            for (int rr = ty; rr < TH + 2 * WH; rr += 8) {
                const int r = rbase - WH + rr;
                tile[rr][tx] = (r >= 0 && r < a.H && x < a.Wp) ? __ldg(src + (size_t)r * a.Wp + x) : 0.f;
            }
            __syncthreads();
            float win[RPT + 2 * WH];
#pragma unroll
            for (int j = 0; j < RPT + 2 * WH; ++j) win[j] = tile[ty * RPT + j][tx];
            float y[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                float acc = g.g[0] * win[j + WH];
#pragma unroll
                for (int dd = 1; dd <= WH; ++dd) acc = fmaf(g.g[dd], win[j + WH - dd] + win[j + WH + dd], acc);
                y[j] = acc;
            }
            cb.step(k, a.N, P.s2, y);
        }
    }
    int nonpos = 0;
    AdjSums sums = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = rbase + ty * RPT + j;
        if (r < a.H && x < a.W) finish_pixel<RPT, MODE>(a, P, plane, r, x, cb, j, nonpos, sums);
    }
    if (MODE == MODE_ADJ) {
        flush_sums(a, plane, sums);
    } else {
        count_nonpos(a.status, nonpos);
    }
}

// Fused forward for the FIR operator (Eq. (8) with the window of Eq. (1)), or
// with BOXP > 0 for the box variant (BOXP passes of a flat kernel of
// half-width WH / BOXP, by running sums: about 2 BOXP additions per sample
// plus one window sum per 8 (rows) or TH / 8 (columns) samples, instead of
// 2 WH + 1 multiply-adds):
// one CTA computes a TH x 32 output tile (TH rows: 16, 32 or 64) for all K
// channels without writing the row-filtered planes.  Per channel k (ascending):
//   1. Phi_k = 2^e0 E u^k on the tile plus a WH halo (zero outside the image),
//      by one multiply per sample from the previous channel, into shared memory;
//   2. row filter of the (TH + 2 WH) rows x 32 columns (work items: row x strip of 8);
//   3. column filter of the TH x 32 outputs (threads: column x TH / 8 rows), times beta_k,
//      accumulated with running powers of u:
//        p += k u^{k-1} Psi_k,  q += u^{k-1} Psi_k (1 <= k <= N),  Psi_0 kept;
//   y = t_c + R p / (Psi_0 + s^2 u q).
// A taller tile shares its halo columns among more outputs; a shorter one
// gives small images more CTAs.  The row-filtered tile is double-buffered by
// channel parity, so each channel costs two barriers.
// grid (ceil(W/32), ceil(H/TH), planes), block 256.
// Sum over j of win[j .. j + 2 R] for the LOUT outputs after BOXP passes of a
// box of half-width R (running sums; each pass shortens the window by 2 R).
template <int BOXP, int R, int LOUT>
__device__ __forceinline__ void box_passes(const float *win, float *out)
{
    constexpr int L0 = LOUT + 2 * BOXP * R;
    float cur[L0];
#pragma unroll
    for (int j = 0; j < L0; ++j) cur[j] = win[j];
#pragma unroll
    for (int p = 0; p < BOXP; ++p) {
        const int lin = L0 - 2 * R * p, lout = lin - 2 * R;
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i <= 2 * R; ++i) acc += cur[i];
        float nxt[L0];
        nxt[0] = acc;
#pragma unroll
        for (int j = 1; j < L0; ++j) {
            if (j < lout) {
                acc += cur[j + 2 * R] - cur[j - 1];
                nxt[j] = acc;
            }
        }
#pragma unroll
        for (int j = 0; j < L0; ++j)
            if (j < lout) cur[j] = nxt[j];
    }
#pragma unroll
    for (int j = 0; j < LOUT; ++j) out[j] = cur[j];
}

template <int WH, int BOXP = 0, int TH = 32>
__global__ void __launch_bounds__(256) fir_fused(ColArgs a, FIRCoef g)
{
    static_assert(TH == 16 || TH == 32 || TH == 64, "tile heights 16, 32, 64");
    constexpr int T = 32;                          // tile width
    constexpr int RPT = TH / 8;                    // output rows per thread
    constexpr int RSW = T + 2 * WH, RSH = TH + 2 * WH;  // tile plus halo
    constexpr int NR = (RSH * RSW + 255) / 256;    // halo samples per thread
    __shared__ float phi[RSH][RSW + 1];
    __shared__ float rf[2][RSH][T + 1];
    const int tid = threadIdx.x;
    const int plane = blockIdx.z;
    const int x0 = blockIdx.x * T, y0 = blockIdx.y * TH;
    const PlaneParams &P = a.pp[plane];
    const float *fp = a.f + (size_t)plane * a.H * a.pitch;
    // output pixels of this thread: column c, rows r0 .. r0 + RPT - 1
    const int c = tid & 31, r0 = (tid >> 5) * RPT;
    const int xo = x0 + c;
    if (P.mode != 0) {  // constant plane or non-finite input: the result is the input
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int yo = y0 + r0 + j;
            if (yo < a.H && xo < a.W) {
                const size_t pix = ((size_t)plane * a.H + yo) * a.pitch + xo;
                a.y[pix] = __ldg(a.f + pix);
            }
        }
        return;
    }
    float hu[NR], hv[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int idx = tid + 256 * i;
        const int rr = idx / RSW, cc = idx % RSW;
        const int gy = y0 - WH + rr, gx = x0 - WH + cc;
        const bool in = idx < RSH * RSW && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
        const float uu = in ? (__ldg(fp + (size_t)gy * a.pitch + gx) - P.tc) * P.invR : 0.f;
        hu[i] = uu;
        hv[i] = in ? envelope(P, uu) : 0.f;
    }
    float ou[RPT], pacc[RPT], qacc[RPT], psi0[RPT], w[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int yo = y0 + r0 + j;
        const bool in = yo < a.H && xo < a.W;
        ou[j] = in ? (__ldg(fp + (size_t)yo * a.pitch + xo) - P.tc) * P.invR : 0.f;
        pacc[j] = qacc[j] = psi0[j] = 0.f;
        w[j] = 1.f;
    }
    // row-filter work items: row rr, columns 8 s .. 8 s + 7 (RSH x 4 items, 256 at a time)
#pragma unroll 1
    for (int k = 0; k < a.K; ++k) {
        const int buf = k & 1;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int idx = tid + 256 * i;
            if (k > 0) hv[i] *= hu[i];
            if (idx < RSH * RSW) phi[idx / RSW][idx % RSW] = hv[i];
        }
        __syncthreads();  // Phi_k on the halo tile; every thread is past the row filter of channel k - 1
#pragma unroll
        for (int item = tid; item < 4 * RSH; item += 256) {
            const int rr_row = item >> 2, cs = (item & 3) * 8;
            float win[8 + 2 * WH];
#pragma unroll
            for (int j = 0; j < 8 + 2 * WH; ++j) win[j] = phi[rr_row][cs + j];
            if constexpr (BOXP > 0) {
                float o8[8];
                box_passes<BOXP, WH / (BOXP > 0 ? BOXP : 1), 8>(win, o8);
#pragma unroll
                for (int j = 0; j < 8; ++j) rf[buf][rr_row][cs + j] = o8[j];
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float acc = g.g[0] * win[j + WH];
#pragma unroll
                    for (int dd = 1; dd <= WH; ++dd) acc = fmaf(g.g[dd], win[j + WH - dd] + win[j + WH + dd], acc);
                    rf[buf][rr_row][cs + j] = acc;
                }
            }
        }
        __syncthreads();  // row-filtered tile of channel k
        float win[RPT + 2 * WH];
#pragma unroll
        for (int j = 0; j < RPT + 2 * WH; ++j) win[j] = rf[buf][r0 + j][c];
        const float beta = P.beta[k];
        const float mk = (float)k;
        float o4[RPT];
        if constexpr (BOXP > 0) {
            box_passes<BOXP, WH / (BOXP > 0 ? BOXP : 1), RPT>(win, o4);
        } else {
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                float acc = g.g[0] * win[j + WH];
#pragma unroll
                for (int dd = 1; dd <= WH; ++dd) acc = fmaf(g.g[dd], win[j + WH - dd] + win[j + WH + dd], acc);
                o4[j] = acc;
            }
        }
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const float psi = o4[j] * beta;
            if (k == 0) {
                psi0[j] = psi;
            } else {
                pacc[j] = fmaf(mk * w[j], psi, pacc[j]);
                if (k <= a.N) qacc[j] = fmaf(w[j], psi, qacc[j]);
                w[j] *= ou[j];
            }
        }
    }
    bool nonpos = false;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int yo = y0 + r0 + j;
        if (yo < a.H && xo < a.W) {
            const float Q = fmaf(P.s2 * ou[j], qacc[j], psi0[j]);
            float out;
            if (!(Q > 0.f)) {  // rare: counted one pixel at a time; the pixel keeps its value
                nonpos = true;
                atomicAdd(status_counters(a.status), 1ull);
                out = __ldg(a.f + ((size_t)plane * a.H + yo) * a.pitch + xo);
            } else {
                out = fmaf(P.R, __fdiv_rn(pacc[j], Q), P.tc);
            }
            a.y[((size_t)plane * a.H + yo) * a.pitch + xo] = out;
        }
    }
    if (__any_sync(0xffffffffu, nonpos) && (tid & 31) == 0) atomicOr(a.status, 0x1u);
}

// Backward finish: dL/df = dL/dh + (sum dL/dy - sum dL/dh) / |I| when the
// centre is the plane mean (Algorithm 1 step 1), and dL/dsigma_r per plane
// = dL/d(s^2) * d(s^2)/dsigma_r = dL/d(s^2) * (-2 s^2 / sigma_r).
// grid (ceil(H*W / 256), planes), block 256.
// grid (row bands, planes), block 256: the centring term of the gradient and
// dL/dsigma_r.  The per-plane shift is formed once per block (one FP64
// division) and added along the band's rows.
__global__ void __launch_bounds__(256) grad_finish(float *__restrict__ grad, const double *__restrict__ acc,
                                                   const PlaneParams *__restrict__ pp, int H, int W, int pitch,
                                                   int centre_mean, double sigma_r, float *__restrict__ grad_sigma_r)
{
    const int plane = blockIdx.y;
    const double *ac = acc + plane * NACC;
    __shared__ float sh_shift;
    if (threadIdx.x == 0) {
        sh_shift = centre_mean ? (float)((ac[0] - ac[1]) / ((double)H * (double)W)) : 0.f;
        if (blockIdx.x == 0 && grad_sigma_r) {
            const double s2 = (double)pp[plane].s2;
            grad_sigma_r[plane] = (s2 > 0.0 && pp[plane].mode == 0 && !isinf(sigma_r))
                                      ? (float)(ac[2] * (-2.0 * s2 / sigma_r))
                                      : 0.f;
        }
    }
    __syncthreads();
    const float shift = sh_shift;
    const int rows = (H + (int)gridDim.x - 1) / (int)gridDim.x;
    const int r0 = blockIdx.x * rows, r1 = min(H, r0 + rows);
    float *g = grad + (size_t)plane * H * pitch;
    for (int r = r0; r < r1; ++r)
        for (int c = threadIdx.x; c < W; c += blockDim.x) g[(size_t)r * pitch + c] += shift;
}

// ------------------------------------------------------------------ tensor-core passes
//
// The same recursive filter with the chunk-local work done by warp-level
// tensor-core products (mma.sync m16n8k8, TF32 inputs, FP32 accumulation).
// Chunks are C = 8 samples.  For a group of 16 chunks X (16 x 8, one chunk per
// row):
//   Y  = X Mloc        Mloc[k][n] = h(|n - k|)          (both recursions inside the chunk)
//   S  = X Msum        chunk end states, 4 combos x (re, im): combo 0/1 causal
//                      pole 0/1 (sum_k p^{7-k} x_k), combo 2/3 anticausal
//                      pole 0/1 (sum_k p^k x_k); column 2c + {0 re, 1 im}
//   Y += Cr Mcor       Cr = incoming states (16 x 8: entry c = Re, c + 4 = Im of
//                      combo c), Mcor[c][n] = Re(A p^{n+1}), Mcor[c+4][n] = -Im(A p^{n+1})
//                      for causal combos and A p^{8-n} for anticausal ones
// Each product runs as three TF32 products (hi*hi + lo*hi + hi*lo, the data
// and the matrices split into a TF32 high part and the TF32 rounding of the
// remainder), which keeps FP32-level accuracy.  The states between chunks are
// combined with the modal scan as before (carry across a chunk = p^8).
// In the fragment layout, thread (g = lane/4, t = lane%4) holds, for the
// chunks of MMA rows g and g + 8, exactly the (Re, Im) of combo t in S and
// the entries t, t + 4 of Cr: the scan of combo t runs in the thread that
// needs its result.

constexpr int TC_C = 8;

struct TCMat {
    float loc[8][8];  // [k][n]
    float sum[8][8];  // [k][s]
    float cor[8][8];  // [e][n]
};

// x = hi + lo with hi = x rounded to its leading 11 significant bits (exact in
// TF32) and lo = x - hi (exact in FP32), of which the tensor core uses the
// leading 11 bits: |x - hi - lo_tf32| < 2^-22 |x|.  The rounding is done on
// the bit pattern: adding half of the 13 dropped mantissa bits' range rounds
// the magnitude half away from zero (carrying into the exponent when the kept
// bits overflow), the mask drops them.  Two integer operations and one FP32
// subtraction; x must be finite and below 2^127 in magnitude.
__device__ __forceinline__ unsigned tf32_hi(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }
__device__ __forceinline__ void tf32_split(float x, unsigned &hi, unsigned &lo)
{
    hi = tf32_hi(x);
    lo = __float_as_uint(__fsub_rn(x, __uint_as_float(hi)));
}
// The same split on the FMA pipe (Veltkamp, constant 2^13 + 1: hi = c - (c - x)
// with c = (2^13 + 1) x keeps the leading 11 bits, rounded to nearest), for a
// kernel whose integer pipe is the busier one.  Every step must round on its
// own: a contracted multiply-subtract would skip the rounding of c.
__device__ __forceinline__ void tf32_split_fma(float x, unsigned &hi, unsigned &lo)
{
    const float c = __fmul_rn(x, 8193.f);
    const float h = __fsub_rn(c, __fsub_rn(c, x));
    hi = __float_as_uint(h);
    lo = __float_as_uint(__fsub_rn(x, h));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// B fragment of an 8 x 8 matrix for this lane, split: b0 = B[t][g], b1 = B[t+4][g]
struct BFrag {
    unsigned h0, h1, l0, l1;
    __device__ __forceinline__ void load(const float (&B)[8][8], int g, int t)
    {
        tf32_split(B[t][g], h0, l0);
        tf32_split(B[t + 4][g], h1, l1);
    }
};

// d += A B in three TF32 products; A given as four FP32 values (fragment order)
__device__ __forceinline__ void mma3(float (&d)[4], float a0, float a1, float a2, float a3, const BFrag &b)
{
    unsigned h0, h1, h2, h3, l0, l1, l2, l3;
    tf32_split(a0, h0, l0);
    tf32_split(a1, h1, l1);
    tf32_split(a2, h2, l2);
    tf32_split(a3, h3, l3);
    mma_tf32(d, l0, l1, l2, l3, b.h0, b.h1);
    mma_tf32(d, h0, h1, h2, h3, b.l0, b.l1);
    mma_tf32(d, h0, h1, h2, h3, b.h0, b.h1);
}

// A fragment split once into TF32 high and low parts, reused by several products
struct AFrag {
    unsigned h0, h1, h2, h3, l0, l1, l2, l3;
    template <bool FMA_PIPE = false>
    __device__ __forceinline__ void set(float a0, float a1, float a2, float a3)
    {
        if (FMA_PIPE) {
            tf32_split_fma(a0, h0, l0);
            tf32_split_fma(a1, h1, l1);
            tf32_split_fma(a2, h2, l2);
            tf32_split_fma(a3, h3, l3);
            return;
        }
        h0 = tf32_hi(a0);
        h1 = tf32_hi(a1);
        h2 = tf32_hi(a2);
        h3 = tf32_hi(a3);
        float r0, r1, r2, r3;  // the remainders, two exact subtractions per instruction
        sub2(r0, r1, a0, a1, __uint_as_float(h0), __uint_as_float(h1));
        sub2(r2, r3, a2, a3, __uint_as_float(h2), __uint_as_float(h3));
        l0 = __float_as_uint(r0);
        l1 = __float_as_uint(r1);
        l2 = __float_as_uint(r2);
        l3 = __float_as_uint(r3);
    }
};

// d += A B as three TF32 products (lo*hi, hi*lo, hi*hi)
__device__ __forceinline__ void mma3f(float (&d)[4], const AFrag &a, const BFrag &b)
{
    mma_tf32(d, a.l0, a.l1, a.l2, a.l3, b.h0, b.h1);
    mma_tf32(d, a.h0, a.h1, a.h2, a.h3, b.l0, b.l1);
    mma_tf32(d, a.h0, a.h1, a.h2, a.h3, b.h0, b.h1);
}

// The lane's combo walks its 8 chunks forwards (causal) or backwards
// (anticausal).  To keep every lane on the same instructions, the 8 (Re, Im)
// chunk values are first copied into scan order with selects (compile-time
// register indices on both sides), scanned forwards, and copied back.
//   S[q][2h], S[q][2h+1]: Re, Im of chunk c = 2q + h.
struct Seq8 {
    float r[8], i[8];
    __device__ __forceinline__ void from_chunks(const float (&S)[4][4], bool rev)
    {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int c = s, cr = 7 - s;
            r[s] = rev ? S[cr >> 1][2 * (cr & 1)] : S[c >> 1][2 * (c & 1)];
            i[s] = rev ? S[cr >> 1][2 * (cr & 1) + 1] : S[c >> 1][2 * (c & 1) + 1];
        }
    }
};

// Row pass, tensor cores.  Each warp filters 512 consecutive samples (64
// chunks) of one row; a row of W samples uses wpr = next_pow2(ceil(W/512))
// warps, a CTA holds 256 / (32 wpr) rows (one row of 512 threads when
// wpr = 16).  Thread (g, t) owns chunks 8g .. 8g+7 of its warp: in group q
// the MMA row g is chunk 8g + 2q and row g + 8 chunk 8g + 2q + 1.  The chunk
// scan of combo t runs in registers over those 8 chunks, then across the 8
// threads g of the warp (shuffles), then across the warps of the row.
// grid (ceil(H / rows_per_cta), planes).
template <int MODE>
__device__ __forceinline__ void row_tc_body(const RowArgs &a, const IIRCoef &cf, const TCMat &tm, int grp,
                                            int plane)
{
    // [channel parity][warp][combo] warp totals: a thread writes the slot of channel k + 2 only after
    // every thread has passed the barrier of channel k + 1, so one barrier per channel suffices
    __shared__ float2 wtot[2][16][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wpr = a.T;  // warps per row
    const int rows_per_cta = (blockDim.x >> 5) / wpr;
    const int r_local = warp / wpr, wr = warp % wpr;
    const int row = grp * rows_per_cta + r_local;
    const bool rv = row < a.H;
    const PlaneParams &P = a.pp[plane];
    if (MODE == MODE_ADJ && grp == 0) zero_acc(a, plane);
    if (P.mode != 0) return;

    // sample of group q, fragment slot i: a0 = chunk 8g+2q sample t, a1 = chunk 8g+2q+1 sample t,
    // a2 = chunk 8g+2q sample t+4, a3 = chunk 8g+2q+1 sample t+4
    const int xw = wr * 512 + 64 * g;
    auto pos = [&](int q, int i) { return xw + 16 * q + t + (i == 1 ? 8 : i == 2 ? 4 : i == 3 ? 12 : 0); };
    RowGen<16, MODE> gen;
    {
        const float *frow = a.f + ((size_t)plane * a.H + (rv ? row : 0)) * a.pitch;
        gen.s2 = P.s2;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int x = pos(q, i);
                const int j = q * 4 + i;
                const bool in = rv && x < a.W;
                const float fv = in ? __ldg(frow + x) : P.tc;
                const float uu = (fv - P.tc) * P.invR;
                gen.u[j] = in ? uu : 0.f;
                if (MODE != MODE_ADJ) {
                    gen.v[j] = in ? envelope(P, uu) : 0.f;
                    gen.t[j] = 0.f;
                } else {
                    float al = 0.f, rho = 0.f;
                    if (in) {
                        const float gyv = __ldg(a.gy + ((size_t)plane * a.H + row) * a.pitch + x);
                        const float Pt = __ldg(a.saved + saved_idx(plane, 0, a.H, a.W, row, x));
                        const float Qt = __ldg(a.saved + saved_idx(plane, 1, a.H, a.W, row, x));
                        if (Qt > 0.f && isfinite(gyv)) {
                            al = __fdiv_rn(gyv * P.R, Qt);
                            rho = __fdiv_rn(Pt, Qt);
                        }
                    }
                    gen.v[j] = al;
                    gen.t[j] = rho;
                }
            }
    }
    BFrag bl, bs, bc;
    bl.load(tm.loc, g, t);
    bs.load(tm.sum, g, t);
    bc.load(tm.cor, g, t);
    const int m = t & 1;
    const bool rev = (t >> 1) != 0;  // anticausal combo: scan order reversed
    const int jpos = rev ? 7 - g : g;  // this thread's place in the warp's scan order
    const float P1r = cf.Pr[m][0], P1i = cf.Pi[m][0];  // p^8: one chunk
    float Pjr, Pji;                                    // p^{64 jpos}: the warp carry reaches this thread
    cpow_tab(Pjr, Pji, cf, m, 8 * jpos);
    float *orow = a.ws + ((size_t)plane * a.K * a.H + (rv ? row : 0)) * a.Wp;
    // The carry entering warp wr from the other warps of the row is
    // sum_w p^{512 d_w} T_w over the warp totals T_w that precede it in scan
    // order, d_w = wr - 1 - w (causal) or w - wr - 1 (anticausal).  Thread g
    // takes the terms of warps g and g + 8 (weight 0 where w does not precede
    // wr); the 8 threads of the combo add them up.
    // (the adjoint, whose channel generator holds more state, folds the totals
    // serially instead and keeps no weights in registers; it also splits its
    // TF32 operands on the FMA pipe: both measured faster for it)
    float Q0r = 0.f, Q0i = 0.f, Q1r = 0.f, Q1i = 0.f;
#pragma unroll
    for (int h = 0; h < (MODE == MODE_ADJ ? 0 : 2); ++h) {
        const int w = g + 8 * h;
        const int d = rev ? w - wr - 1 : wr - 1 - w;
        if (w < wpr && d >= 0) {
            float qr, qi;
            cpow_tab(qr, qi, cf, m, 64 * d);
            if (h == 0) {
                Q0r = qr;
                Q0i = qi;
            } else {
                Q1r = qr;
                Q1i = qi;
            }
        }
    }

#pragma unroll 1
    for (int k = 0; k < a.K; ++k) {
        float x16[16];
        gen.channel(k, a.N, x16);
        float D[4][4], S[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int i = 0; i < 4; ++i) D[q][i] = S[q][i] = 0.f;
            AFrag af;
            af.template set<MODE == MODE_ADJ>(x16[4 * q], x16[4 * q + 1], x16[4 * q + 2], x16[4 * q + 3]);
            mma3f(D[q], af, bl);
            mma3f(S[q], af, bs);
        }
        Seq8 sq;
        sq.from_chunks(S, rev);
        // the thread's 8 chunks from zero state
        float vr = 0.f, vi = 0.f;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            float nr = sq.r[s], ni = sq.i[s];
            cmadd(nr, ni, P1r, P1i, vr, vi);
            vr = nr;
            vi = ni;
        }
        // across the 8 threads g of the warp, in scan order (p^{64 d} per d threads)
#pragma unroll
        for (int st = 0; st < 3; ++st) {
            const int d = 1 << st;
            const int src = 4 * (rev ? g + d : g - d) + t;
            const float ur = __shfl_sync(0xffffffffu, vr, src & 31);
            const float ui = __shfl_sync(0xffffffffu, vi, src & 31);
            if (jpos >= d) cmadd(vr, vi, cf.Pr[m][st + 3], cf.Pi[m][st + 3], ur, ui);
        }
        const int srcx = 4 * (rev ? g + 1 : g - 1) + t;
        float er = __shfl_sync(0xffffffffu, vr, srcx & 31);
        float ei = __shfl_sync(0xffffffffu, vi, srcx & 31);
        if (jpos == 0) er = ei = 0.f;
        if (wpr > 1) {
            const int last = 4 * (rev ? 0 : 7) + t;
            const float wtr = __shfl_sync(0xffffffffu, vr, last), wti = __shfl_sync(0xffffffffu, vi, last);
            const int par = k & 1;
            if (g == 0) wtot[par][warp][t] = make_float2(wtr, wti);
            __syncthreads();
            const int w0 = r_local * wpr;
            float Wr = 0.f, Wi = 0.f;
            if constexpr (MODE == MODE_ADJ) {
                const float pwr = cf.Pr[m][6], pwi = cf.Pi[m][6];  // p^512: one warp
                for (int s = 0; s < wpr; ++s) {
                    const int w = rev ? wpr - 1 - s : s;
                    if ((!rev && w >= wr) || (rev && w <= wr)) continue;
                    const float2 tt = wtot[par][w0 + w][t];
                    float nr = tt.x, ni = tt.y;
                    cmadd(nr, ni, pwr, pwi, Wr, Wi);
                    Wr = nr;
                    Wi = ni;
                }
            } else {
                {
                    // warps g >= wpr read the row's last total (written, finite) with weight 0
                    const float2 tt = wtot[par][w0 + min(g, wpr - 1)][t];
                    cmul(Wr, Wi, Q0r, Q0i, tt.x, tt.y);
                }
                if (wpr > 8) {
                    const float2 tt = wtot[par][w0 + g + 8][t];
                    cmadd(Wr, Wi, Q1r, Q1i, tt.x, tt.y);
                }
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {
                    Wr += __shfl_xor_sync(0xffffffffu, Wr, o);
                    Wi += __shfl_xor_sync(0xffffffffu, Wi, o);
                }
            }
            cmadd(er, ei, Pjr, Pji, Wr, Wi);
        }
        // incoming state of each chunk, in scan order, then back to chunk order
        float inr_s[8], ini_s[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            inr_s[s] = er;
            ini_s[s] = ei;
            float nr = sq.r[s], ni = sq.i[s];
            cmadd(nr, ni, P1r, P1i, er, ei);
            er = nr;
            ei = ni;
        }
        const float beta = P.beta[k];
        float *o = orow + (size_t)k * a.H * a.Wp;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c0 = 2 * q, c1 = 2 * q + 1;
            const float r0 = rev ? inr_s[7 - c0] : inr_s[c0], i0 = rev ? ini_s[7 - c0] : ini_s[c0];
            const float r1 = rev ? inr_s[7 - c1] : inr_s[c1], i1 = rev ? ini_s[7 - c1] : ini_s[c1];
            AFrag cfr;
            cfr.template set<MODE == MODE_ADJ>(r0, r1, i0, i1);
            mma3f(D[q], cfr, bc);
            if (rv) {
                const int xa = xw + 16 * q + 2 * t, xb = xa + 8;
                float2 oa, ob;
                mul2(oa.x, oa.y, D[q][0], D[q][1], beta, beta);
                mul2(ob.x, ob.y, D[q][2], D[q][3], beta, beta);
                if (xa + 1 < a.Wp) *reinterpret_cast<float2 *>(o + xa) = oa;
                if (xb + 1 < a.Wp) *reinterpret_cast<float2 *>(o + xb) = ob;
            }
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(512) row_tc(RowArgs a, IIRCoef cf, TCMat tm)
{
    row_tc_body<MODE>(a, cf, tm, blockIdx.x, blockIdx.y);
}

// Column pass, tensor cores (mma.sync, TF32 x 3).  The cluster structure is
// col_iir's: a cluster of CL <= 8 CTAs covers an 8-column strip's full height,
// CTA rank r owns rows [512 r, 512 r + 512); channel tiles are staged by
// cp.async two channels ahead in four buffers; warp 0 turns the warp totals
// into the carry entering each warp and pushes the CTA total, already carried
// across the CTAs in between, into the CTAs it enters; a split cluster barrier
// publishes them.  The products are row_tc's: warp w owns rows
// [64 w, 64 w + 64) of the CTA, 8 chunks of 8 rows per column; in group q its
// MMA row g is (column g, chunk 2q) and row g + 8 is (column g, chunk 2q + 1).
// Thread (g, t) thus holds combo t (pole t & 1, direction t >> 1) of column g
// for the warp's 8 chunks, so the chunk scan runs in its registers, and its 16
// outputs are column g, rows 64 w + 16 q + 8 h + 2 t + {0, 1} (h = 0, 1).
// grid (strips * CL, planes), block 256, cluster (CL, 1, 1).
template <int MODE>
__device__ __forceinline__ void col_tc_body(const ColArgs &a, const IIRCoef &cf, const TCMat &tm, int strip,
                                            int plane)
{
    extern __shared__ __align__(16) float tiles[];  // [COL_TILE_BUFS][COL_TILE_FLOATS], col_iir's tile layout
    // [channel parity][warp][column][combo]: warp totals; warp 0 replaces them by the carry entering each warp
    __shared__ float2 wt[2][8][8][4];
    // [channel parity][source rank][column][combo]: CTA totals pushed by the other CTAs of the cluster
    // (causal combos by lower ranks, anticausal ones by higher ranks), each already carried across the
    // CTAs in between; slots no CTA writes stay zero
    __shared__ float2 inc[2][8][8][4];
    // the B fragments of every lane, split (TF32 high and low parts): loc, sum, cor
    __shared__ uint4 sbf[3][32];
    // forward: u of this thread's pixel pairs (j = 2e, 2e + 1), kept out of registers
    constexpr bool FWD = MODE == MODE_FWD;
    __shared__ float2 su[FWD ? 8 : 1][FWD ? 256 : 1];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int CL = (int)cl.num_blocks();
    const int x = strip * 8 + g;
    const int rbase = rank * COL_ROWS;
    const PlaneParams &P = a.pp[plane];
    const bool filt = (P.mode == 0);
    const float *wsp = a.ws + (size_t)plane * a.K * a.H * a.Wp + strip * 8;

    // tile copy: every warp copies the 64 rows it reads itself (rows 64 w + lane/2 + 16 i, i < 4, two
    // 16-byte halves), so a tile needs no CTA-wide barrier: the warp's own wait and __syncwarp
    const size_t plane_stride = (size_t)a.H * a.Wp;
    const int lrow = 64 * warp + (lane >> 1);
    const int gr0 = rbase + lrow;
    const int src0 = gr0 * a.Wp + (lane & 1) * 4;
    const unsigned dst0 = smem_u32(tiles + tile_off(lrow) + (lane & 1) * 4);
    auto issue_tile = [&](int k) {
        const float *src = wsp + (size_t)k * plane_stride + src0;
        const unsigned dst = dst0 + (unsigned)((k & (COL_TILE_BUFS - 1)) * COL_TILE_FLOATS * sizeof(float));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool ok = filt && gr0 + 16 * i < a.H;
            // tile_off(r + 16) = tile_off(r) + 17 * 8
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst + i * 17 * 8 * 4),
                         "l"(ok ? src + (size_t)i * 16 * a.Wp : wsp), "r"(ok ? 16 : 0)
                         : "memory");
        }
    };

    // pixel j = 4 q + i of this thread: row 64 w + 16 q + 8 (i >> 1) + 2 t + (i & 1) of the CTA
    auto prow = [&](int q, int i) { return rbase + 64 * warp + 16 * q + 8 * (i >> 1) + 2 * t + (i & 1); };
    // the per-pixel sums: for the forward p and q in registers and u in shared memory (the same
    // Horner steps as Combine), otherwise Combine
    Combine<16, MODE> cb;
    float fp[FWD ? 16 : 1], fq[FWD ? 16 : 1];
    const float *fcol = a.f + (size_t)plane * a.H * a.pitch;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = prow(q, i);
            const bool in = (r < a.H) && (x < a.W);
            const float fv = in ? __ldg(fcol + (size_t)r * a.pitch + x) : 0.f;
            const float uu = (fv - P.tc) * P.invR;
            if constexpr (FWD) {
                const int j = q * 4 + i;
                if (j & 1)
                    su[j >> 1][tid].y = uu;
                else
                    su[j >> 1][tid].x = uu;
                fp[j] = fq[j] = 0.f;
            } else {
                cb.init(uu, q * 4 + i);
            }
        }
    if (tid < 32) {
        BFrag b;
        b.load(tm.loc, g, t);
        sbf[0][lane] = make_uint4(b.h0, b.h1, b.l0, b.l1);
        b.load(tm.sum, g, t);
        sbf[1][lane] = make_uint4(b.h0, b.h1, b.l0, b.l1);
        b.load(tm.cor, g, t);
        sbf[2][lane] = make_uint4(b.h0, b.h1, b.l0, b.l1);
    }
    auto bfrag = [&](int which) {
        const uint4 v = sbf[which][lane];
        BFrag b;
        b.h0 = v.x;
        b.h1 = v.y;
        b.l0 = v.z;
        b.l1 = v.w;
        return b;
    };
    const int m = t & 1;
    const bool rev = (t >> 1) != 0;                      // anticausal combo: scan order reversed
    const float P1r = cf.Pr[m][0], P1i = cf.Pi[m][0];    // p^8: one chunk
    float Phr, Phi;  // p^{64 w'}: a carry from outside the CTA crosses the warps before (causal) / after this one
    cpow_tab(Phr, Phi, cf, m, 8 * (rev ? 7 - warp : warp));
    {
        float2 *z = &inc[0][0][0][0];
        for (int e = tid; e < 2 * 8 * 8 * 4; e += blockDim.x) z[e] = make_float2(0.f, 0.f);
    }
    cl.sync();  // zeroed before any peer pushes

    issue_tile(a.K - 1);
    cp_async_commit();
    if (a.K >= 2) issue_tile(a.K - 2);
    cp_async_commit();
    cp_async_wait_1();
    __syncthreads();
    // this warp's rows in a tile: tile_off(64 w + 16 q + r) = (68 w + 17 q + r) * 8 for r < 16
    const int toff = 68 * 8 * warp + g;
    // the A values of the next channel's tile, loaded as soon as the tile is visible
    float xa[4][4];
    auto load_a = [&](int k) {
        const float *tl = tiles + (k & (COL_TILE_BUFS - 1)) * COL_TILE_FLOATS + toff;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float *tq = tl + 17 * 8 * q;
            xa[q][0] = tq[t * 8];
            xa[q][1] = tq[(t + 8) * 8];
            xa[q][2] = tq[(t + 4) * 8];
            xa[q][3] = tq[(t + 12) * 8];
        }
    };
    load_a(a.K - 1);
#pragma unroll 1
    for (int k = a.K - 1; k >= 0; --k) {
        // tile k's A values are in xa (loaded after the warp's copies landed); the buffer of tile
        // k - 2 last held tile k + 2, which this warp finished reading before issuing this copy
        float D[4][4], S[4][4];
        const BFrag bl = bfrag(0), bs = bfrag(1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            AFrag af;
            af.set(xa[q][0], xa[q][1], xa[q][2], xa[q][3]);
#pragma unroll
            for (int i = 0; i < 4; ++i) D[q][i] = S[q][i] = 0.f;
            mma3f(D[q], af, bl);
            mma3f(S[q], af, bs);
        }
        if (k >= 2) issue_tile(k - 2);
        cp_async_commit();

        // the warp total of combo t of column g (zero state at the warp's start, in scan order)
        Seq8 sq;
        sq.from_chunks(S, rev);
        float tr = 0.f, ti = 0.f;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            float nr = sq.r[s], ni = sq.i[s];
            cmadd(nr, ni, P1r, P1i, tr, ti);
            tr = nr;
            ti = ni;
        }
        const int par = k & 1;
        wt[par][warp][g][t] = make_float2(tr, ti);
        if (warp == 0) {
            bar_sync_named(1, 256);  // all warp totals of this channel written
            // lane (g, t): fold the 8 warp totals in scan order; each slot becomes the carry entering its warp
            const float P8r = m == 0 ? cf.Pr[0][3] : cf.Pr[1][3], P8i = m == 0 ? cf.Pi[0][3] : cf.Pi[1][3];  // p^64
            float Wr = 0.f, Wi = 0.f;
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int w = rev ? 7 - s : s;
                const float2 tt = wt[par][w][g][t];
                wt[par][w][g][t] = make_float2(Wr, Wi);
                float nr = tt.x, ni = tt.y;
                cmadd(nr, ni, P8r, P8i, Wr, Wi);
                Wr = nr;
                Wi = ni;
            }
            // push the CTA total to the CTAs it enters, later ranks (causal) or earlier ones
            // (anticausal), times p^512 per CTA crossed on the way
            float2 *own = &inc[par][rank][g][t];
            const int nd = rev ? rank : CL - 1 - rank;
            const float P64r = m == 0 ? cf.Pr[0][6] : cf.Pr[1][6], P64i = m == 0 ? cf.Pi[0][6] : cf.Pi[1][6];  // p^512
            for (int d = 1; d <= nd; ++d) {
                *cl.map_shared_rank(own, rev ? rank - d : rank + d) = make_float2(Wr, Wi);
                float nr, ni;
                cmul(nr, ni, P64r, P64i, Wr, Wi);
                Wr = nr;
                Wi = ni;
            }
        } else {
            bar_arrive_named(1, 256);
        }
        cp_async_wait_1();  // this thread's part of tile k - 1
        __syncwarp();       // the warp's rows of tile k - 1 visible to the warp
        // releases the carries and the pushed CTA totals
        cluster_arrive_release();
        cluster_wait_acquire();
        if (k >= 1) load_a(k - 1);  // their latency runs under the rest of channel k

        // the carry entering this warp: from the warps before it in the CTA, and from the other CTAs
        float Wr, Wi;
        {
            const float2 w2 = wt[par][warp][g][t];
            Wr = w2.x;
            Wi = w2.y;
        }
        if (CL > 1) {
            float Xr = 0.f, Xi = 0.f;
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const float2 tt = inc[par][s][g][t];
                Xr += tt.x;
                Xi += tt.y;
            }
            cmadd(Wr, Wi, Phr, Phi, Xr, Xi);
        }
        // incoming state of each chunk in scan order (written over the chunk sums), then the
        // correction products in chunk order
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            float nr = sq.r[s], ni = sq.i[s];
            sq.r[s] = Wr;
            sq.i[s] = Wi;
            cmadd(nr, ni, P1r, P1i, Wr, Wi);
            Wr = nr;
            Wi = ni;
        }
        const BFrag bc = bfrag(2);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c0 = 2 * q, c1 = 2 * q + 1;
            const float r0 = rev ? sq.r[7 - c0] : sq.r[c0], i0 = rev ? sq.i[7 - c0] : sq.i[c0];
            const float r1 = rev ? sq.r[7 - c1] : sq.r[c1], i1 = rev ? sq.i[7 - c1] : sq.i[c1];
            AFrag cfr;
            cfr.set(r0, r1, i0, i1);
            mma3f(D[q], cfr, bc);
        }
        float y16[16];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int i = 0; i < 4; ++i) y16[4 * q + i] = D[q][i];
        if constexpr (FWD) {
            // Combine::step of the forward, u from shared memory
            if (k == 0) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float2 uu = su[e][tid];
                    fq[2 * e] = fmaf(P.s2 * uu.x, fq[2 * e], y16[2 * e]);
                    fq[2 * e + 1] = fmaf(P.s2 * uu.y, fq[2 * e + 1], y16[2 * e + 1]);
                }
            } else {
                const float mk = (float)k;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int j = 2 * e;
                    const float2 uu = su[e][tid];
                    if (k <= a.N) fma2r(fq[j], fq[j + 1], uu.x, uu.y, fq[j], fq[j + 1], y16[j], y16[j + 1]);
                    float t0, t1;
                    mul2(t0, t1, mk, mk, y16[j], y16[j + 1]);
                    fma2r(fp[j], fp[j + 1], uu.x, uu.y, fp[j], fp[j + 1], t0, t1);
                }
            }
        } else {
            cb.step(k, a.N, P.s2, y16);
        }
    }
    cl.sync();  // no CTA may leave while a peer can still read its shared memory
    if constexpr (FWD) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float2 uu = su[e][tid];
            cb.u[2 * e] = uu.x;
            cb.u[2 * e + 1] = uu.y;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            cb.p[j] = fp[j];
            cb.q[j] = fq[j];
        }
    }
    int nonpos = 0;
    AdjSums sums = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = prow(q, i);
            if (r < a.H && x < a.W) finish_pixel<16, MODE>(a, P, plane, r, x, cb, 4 * q + i, nonpos, sums);
        }
    if (MODE == MODE_ADJ) {
        flush_sums(a, plane, sums);
    } else {
        count_nonpos(a.status, nonpos);
    }
}

template <int MODE>
__global__ void __launch_bounds__(256, MODE == MODE_SAVE ? 1 : 2) col_tc(ColArgs a, IIRCoef cf, TCMat tm)
{
    col_tc_body<MODE>(a, cf, tm, blockIdx.x / (int)cg::this_cluster().num_blocks(), blockIdx.y);
}

// ------------------------------------------------------------------ batched

// Many planes of different sizes, each with its own sigma_s, sigma_r and
// order, in four launches (stats, finalize, rows, columns), every one of them
// over all planes at once.  The tables below live in the caller's workspace
// (written once by bf_gp_batched_plan_upload); blocks find their plane by a
// binary search over exclusive prefix sums of the planes' work-item counts.
// The recursive filter is used for every plane.
struct BatchPlane {
    const float *f;
    float *y;
    float *ws;  // this plane's K row-filtered planes [K][H][Wp]
    int H, W, pitch, Wp, K, N, T, nblk, rows_per_block, pad;
    double sigma_s, sigma_r;
};

struct BatchArgs {
    const BatchPlane *bp;
    const IIRCoef *coef;  // per plane (chunk length 16 for rows and columns)
    PlaneParams *pp;
    StatPartial *part;
    const int *pre_stats, *pre_rows, *pre_cols;  // n + 1 entries each (pre_cols over the planes in col_order)
    const int *col_order;                        // planes sorted by column cluster size
    uint32_t *status;
    int n, centre_given;
    int cid0;                                    // first (plane, strip) item of this column launch
    int pad;
    double tc_given;
};

__device__ __forceinline__ int find_plane(const int *__restrict__ pre, int n, int id)
{
    int lo = 0, hi = n - 1;  // largest p with pre[p] <= id
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(pre + mid) <= id) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) batched_stats_partial(BatchArgs b)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *b.status = 0u;
    const int p = find_plane(b.pre_stats, b.n, blockIdx.x);
    const BatchPlane &d = b.bp[p];
    stats_partial_body(d.f, d.H, d.W, d.pitch, d.rows_per_block, blockIdx.x - b.pre_stats[p], b.part + blockIdx.x);
}

__global__ void __launch_bounds__(256) batched_stats_finalize(BatchArgs b)
{
    const int p = blockIdx.x;
    const BatchPlane &d = b.bp[p];
    stats_finalize_body(b.part + b.pre_stats[p], d.nblk, (long long)d.H * d.W, b.centre_given, b.tc_given,
                        d.sigma_r, d.sigma_s, d.K, 0, p, b.pp, b.status);
}

// ------------------------------------------------------------------ persistent batched

constexpr int COL_C_PERSIST = 16;  // the column pass's chunk length

// One plane of a persistent batched launch: its buffers, its single-image
// workspace (status word, PlaneParams, statistics partials, channel planes at
// the offsets a single-image call of the same size uses) and its work units.
struct PersistPlane {
    const float *f;
    float *y;
    char *ws;
    long long off_params, off_part, off_planes;
    int H, W, pitch, Wp, K, N, wpr;
    int nblk, rows_per_block, rowgroups, strips;
    int G;  // CTAs per column strip: the power of two >= ceil(H / 512), at most the cluster size
    int stat_m, row_m;  // statistics partials / row groups one CTA takes per item
    double sigma_s, sigma_r;
};

enum { PITEM_STATS = 0, PITEM_FINAL = 1, PITEM_ROWS = 2, PITEM_COLS = 3 };

struct PersistArgs {
    const PersistPlane *pl;
    const IIRCoef *crow;  // per plane: chunk length 8 (tensor-core row pass)
    const TCMat *tm;      // per plane
    const IIRCoef *ccol;  // per plane: chunk length 16 (column pass)
    const int4 *items;    // {kind, plane, first unit, units}, in dependency order
    int *work;            // next item to take (zeroed before the launch)
    int *ready;           // per plane: partials done, finalized, row groups done (zeroed before the launch)
    int nitems, centre_given;
    double tc_given;
    long long wait_cycles;  // budget of one wait for a plane's readiness counter
    int starve_plane;       // testing: this plane's column items wait for one row group more than exists
    int pad;
};

__device__ __forceinline__ int load_acquire(const int *c)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(c) : "memory");
    return v;
}

// Waits until *c >= target (acquire), at most `budget` clock cycles; false if it gave up.
__device__ __forceinline__ bool wait_count(const int *c, int target, long long budget)
{
    const long long t0 = clock64();
    for (;;) {
        const int v = load_acquire(c);
        if (v >= target) return true;
        if (clock64() - t0 > budget) return false;
        __nanosleep(256);
    }
}

// Counts n finished units of a plane: every thread's writes are done, then one release.
__device__ __forceinline__ void count_done(int *c, int n)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(c, n);
    }
}

// The whole batched forward in one launch of resident clusters.  Cluster rank 0
// takes the next item from a counter and hands it to the cluster.  Every item
// comes after the items it needs (all planes' statistics partials, then their
// centres and scales, then the row groups of plane after plane, with each
// plane's column strips placed a few rounds of row items after its last row
// group, so that they find its channel planes still partly in L2), so an item
// only waits for items taken before it, by clusters that are running.  Rank 0
// waits for the item's prerequisite (a per-plane readiness counter, bounded by
// wait_cycles) and the whole cluster follows its decision; a wait that gives up
// raises BF_DEV_TIMEOUT in the plane's status word and the item is skipped (its
// own count still advances, so nothing waits on it in turn).  Statistics and
// row items give stat_m / row_m consecutive units to each CTA; a column item
// gives one strip to each group of G CTAs (the cluster size / G strips at
// once).  Each plane's coefficients are staged in shared memory for its items.
// Same kernels' arithmetic as the single-image forward with engine 0
// (tensor-core rows, CUDA-core columns).  The statuses are zeroed before the
// launch and gathered after it.
// grid (clusters * cluster size), block 256, cluster (size <= 8).
__global__ void __launch_bounds__(256, 2) batched_persistent(PersistArgs a)
{
    __shared__ int s_item, s_go;
    __shared__ IIRCoef s_cf;
    __shared__ TCMat s_tm;
    // the item's arguments, staged like its coefficients: read from shared memory where used
    __shared__ RowArgs s_ra;
    __shared__ ColArgs s_ca;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int CLn = (int)cl.num_blocks();
    const int tid = threadIdx.x;
    auto stage = [&](const void *src, void *dst, int bytes) {
        const int *sp = static_cast<const int *>(src);
        int *dp = static_cast<int *>(dst);
        for (int i = tid; i < bytes / 4; i += blockDim.x) dp[i] = __ldg(sp + i);
    };
    for (;;) {
        if (rank == 0 && tid == 0) s_item = atomicAdd(a.work, 1);
        cl.sync();
        const int it = *cl.map_shared_rank(&s_item, 0);
        if (it >= a.nitems) {
            cl.sync();  // rank 0 leaves only after every peer has read its s_item
            break;
        }
        const int4 w = a.items[it];
        const int p = w.y;
        const PersistPlane &d = a.pl[p];
        int *rdy = a.ready + 3 * p;
        if (rank == 0 && tid == 0) {
            bool go = true;
            if (w.x == PITEM_FINAL) go = wait_count(rdy + 0, d.nblk, a.wait_cycles);
            if (w.x == PITEM_ROWS) go = wait_count(rdy + 1, 1, a.wait_cycles);
            if (w.x == PITEM_COLS) go = wait_count(rdy + 2, d.rowgroups + (p == a.starve_plane), a.wait_cycles);
            s_go = go ? 1 : 0;
            if (!go) {
                uint32_t *status = reinterpret_cast<uint32_t *>(d.ws);
                atomicOr(status, 0x8u);
                atomicAdd(status_counters(status) + 3, 1ull);
            }
        }
        cl.sync();
        const bool go = *cl.map_shared_rank(&s_go, 0) != 0;
        if (go && tid == 0 && w.x != PITEM_STATS) {
            // this CTA's own acquire of the counter rank 0 saw reach its target
            load_acquire(rdy + (w.x == PITEM_FINAL ? 0 : w.x == PITEM_ROWS ? 1 : 2));
        }
        uint32_t *status = reinterpret_cast<uint32_t *>(d.ws);
        PlaneParams *pp = reinterpret_cast<PlaneParams *>(d.ws + d.off_params);
        StatPartial *part = reinterpret_cast<StatPartial *>(d.ws + d.off_part);
        float *planes = reinterpret_cast<float *>(d.ws + d.off_planes);
        if (w.x == PITEM_STATS) {
            // units w.z + rank m .. of the item's w.w, m = stat_m per CTA
            const int u0 = rank * d.stat_m, u1 = min(w.w, u0 + d.stat_m);
            if (u0 < u1) {
                for (int j = u0; j < u1; ++j)
                    stats_partial_body(d.f, d.H, d.W, d.pitch, d.rows_per_block, w.z + j, part + w.z + j);
                count_done(rdy + 0, u1 - u0);
            }
        } else if (w.x == PITEM_FINAL) {
            if (rank == 0) {
                if (go)
                    stats_finalize_body(part, d.nblk, (long long)d.H * d.W, a.centre_given, a.tc_given, d.sigma_r,
                                        d.sigma_s, d.K, 0, 0, pp, status);
                count_done(rdy + 1, 1);
            }
        } else if (w.x == PITEM_ROWS) {
            const int u0 = rank * d.row_m, u1 = min(w.w, u0 + d.row_m);
            if (u0 < u1) {
                stage(a.crow + p, &s_cf, (int)sizeof(IIRCoef));
                stage(a.tm + p, &s_tm, (int)sizeof(TCMat));
                if (tid == 0) {
                    s_ra.f = d.f;
                    s_ra.gy = nullptr;
                    s_ra.fd = nullptr;
                    s_ra.saved = nullptr;
                    s_ra.ws = planes;
                    s_ra.pp = pp;
                    s_ra.acc = nullptr;
                    s_ra.H = d.H;
                    s_ra.W = d.W;
                    s_ra.pitch = d.pitch;
                    s_ra.Wp = d.Wp;
                    s_ra.K = d.K;
                    s_ra.T = d.wpr;
                    s_ra.N = d.N;
                }
                __syncthreads();
                if (go) {
                    for (int j = u0; j < u1; ++j) row_tc_body<MODE_FWD>(s_ra, s_cf, s_tm, w.z + j, 0);
                }
                count_done(rdy + 2, u1 - u0);
            }
        } else {  // PITEM_COLS: every CTA of the cluster, G per strip
            stage(a.ccol + p, &s_cf, (int)sizeof(IIRCoef));
            if (tid == 0) {
                s_ca.ws = planes;
                s_ca.f = d.f;
                s_ca.y = d.y;
                s_ca.gy = nullptr;
                s_ca.saved = nullptr;
                s_ca.pp = pp;
                s_ca.status = status;
                s_ca.acc = nullptr;
                s_ca.H = d.H;
                s_ca.W = d.W;
                s_ca.pitch = d.pitch;
                s_ca.Wp = d.Wp;
                s_ca.K = d.K;
                s_ca.N = d.N;
                s_ca.wait_limit = 0;
                s_ca.no_mma = 0;
            }
            __syncthreads();
            const int G = d.G, g = rank / G;
            const int strip = w.z + g;
            const bool active = go && g < w.w && strip < d.strips;
            col_iir_body<COL_C_PERSIST, MODE_FWD, 8>(s_ca, s_cf, active ? strip : 0, 0, ColGroup{G, rank % G, g * G, active ? 1 : 0});
        }
        __syncthreads();  // the staged coefficients are read before the next item replaces them
    }
}

// Zeroes every plane's status word and counters (before a persistent launch).
__global__ void zero_plane_status(char *ws, const unsigned long long *ofs, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t *st = reinterpret_cast<uint32_t *>(ws + ofs[i]);
        *st = 0u;
        for (int q = 0; q < NCOUNTERS; ++q) status_counters(st)[q] = 0ull;
    }
}

// ORs the status word of every plane's workspace into the batch's (the planes'
// launches have all finished: this kernel follows the join on the stream).
__global__ void gather_status(uint32_t *dst, const char *ws, const unsigned long long *ofs, int n)
{
    // OR of the planes' status words and sums of their counters
    uint32_t bits = 0;
    unsigned long long c[NCOUNTERS] = {};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        bits |= *reinterpret_cast<const uint32_t *>(ws + ofs[i]);
        const unsigned long long *pc = reinterpret_cast<const unsigned long long *>(ws + ofs[i] + 8);
#pragma unroll
        for (int q = 0; q < NCOUNTERS; ++q) c[q] += pc[q];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        bits |= __shfl_down_sync(0xffffffffu, bits, o);
#pragma unroll
        for (int q = 0; q < NCOUNTERS; ++q) c[q] += __shfl_down_sync(0xffffffffu, c[q], o);
    }
    __shared__ uint32_t w[32];
    __shared__ unsigned long long wc[32][NCOUNTERS];
    if ((threadIdx.x & 31) == 0) {
        w[threadIdx.x >> 5] = bits;
#pragma unroll
        for (int q = 0; q < NCOUNTERS; ++q) wc[threadIdx.x >> 5][q] = c[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t b = 0;
        unsigned long long t[NCOUNTERS] = {};
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            b |= w[i];
            for (int q = 0; q < NCOUNTERS; ++q) t[q] += wc[i][q];
        }
        *dst = b;
        for (int q = 0; q < NCOUNTERS; ++q) status_counters(dst)[q] = t[q];
    }
}

}  // namespace bfgp
