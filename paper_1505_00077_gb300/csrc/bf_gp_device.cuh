// bf_gp_device.cuh -- sm_103a kernels of the Gauss-polynomial bilateral filter.
//
// Method: Chaudhury, "Fast and Accurate Bilateral Filtering using
// Gauss-Polynomial Decomposition", Algorithm 1 / Eqs. (7)-(11).
//
// Per plane, with h = f - t_c, R = max|h|, u = h/R, s^2 = (R/sigma_r)^2,
// E = exp(-s^2 u^2/2), channels Phi_k = E u^k (k = 0..K-1, K = N+2) and
// beta_0 = 1, beta_m = s^{2(m-1)}/m! (m >= 1), Psi_k = beta_k * S Phi_k:
//     P~ = sum_{m=1..N+1} m u^{m-1} Psi_m      (= Eq. (9) / (sigma_r s))
//     Q~ = Psi_0 + s^2 u sum_{m=1..N} u^{m-1} Psi_m   (= Eq. (10))
//     y  = t_c + R P~/Q~                        (Eq. (11) + Eq. (6))
// which is Eqs. (9)-(11) after substituting G_n = (s u)^n and
// F_n = s^n Phi_n; P~ is the derivative of the polynomial sum_m v^m Psi_m at
// v = u, so both sums cost 3 FMA per channel and pixel in Horner form.
//
// Kernels (all FP32 arithmetic, IEEE expf and division):
//   stats_partial / stats_finalize : Algorithm 1 step 1 (mean) plus min/max;
//                                    finalize derives t_c, R, s^2, beta (FP64).
//   row_iir / row_fir              : channel generation (steps 2-4, 7, 12) fused
//                                    with the row half of the separable filter
//                                    (steps 8, 13), scaled by beta_k, written
//                                    to the workspace [plane][k][H][Wp].
//   col_iir / col_fir              : column half of the filter fused with the
//                                    combine (steps 11, 14-16) and the division
//                                    (step 18); the column-filtered planes are
//                                    never written.
//
// Recursive filter: Deriche's 4th-order Gaussian (cited in Sec. 3) written as
// h(d) = Re sum_m A_m p_m^d (two complex poles).  The line operator
// y_i = sum_j h(|i-j|) x_j (zero extension) is the sum of a causal part
// (states z_i = x_i + p z_{i-1}, output Re(A z_i)) and an anticausal part
// (states a_i = x_i + p a_{i+1}, output at i: Re(A p a_{i+1})).  A thread owns a
// chunk of C consecutive samples, runs both recursions from zero state, and
// the chunk states are combined by a parallel prefix/suffix scan (carry across
// a chunk = multiply by p^C); the carries enter each output through the
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
    int mode;       // 0 = filter, 1 = copy input to output
    int pad0, pad1;
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
    float pr[NP], pi[NP];                    // poles p_m
    float tr[NP][CMAX + 1], ti[NP][CMAX + 1];  // A_m p_m^e, e = 0..C  (tr[m][0] = Re A_m)
    float Pr[NP][12], Pi[NP][12];            // p_m^{C 2^i}
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

// p^n by binary powering from the table p^{C 2^i}
__device__ __forceinline__ void cpow_tab(float &rr, float &ri, const IIRCoef &cf, int m, int n)
{
    rr = 1.f;
    ri = 0.f;
#pragma unroll 1
    for (int i = 0; i < 12 && n; ++i, n >>= 1)
        if (n & 1) {
            float tr, ti;
            cmul(tr, ti, rr, ri, cf.Pr[m][i], cf.Pi[m][i]);
            rr = tr;
            ri = ti;
        }
}

// Local recursions of one chunk from zero state.
//   y[j]      = sum_m Re(A_m z_j) + Re(A_m p_m a_{j+1})   (a_C = 0)
//   e[m]      = z_{C-1}   (causal state at the chunk end)
//   s[m]      = a_0       (anticausal state at the chunk start)
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
            // causal at j
            const float nzr = fmaf(pr, zr, fmaf(-pi, zi, x[j]));
            const float nzi = fmaf(pr, zi, pi * zr);
            zr = nzr;
            zi = nzi;
            y[j] = fmaf(Ar, zr, fmaf(-Ai, zi, y[j]));
            // anticausal: output at jj uses a_{jj+1}, then a_jj = x_jj + p a_{jj+1}
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

// ------------------------------------------------------------------ stats

// grid (nblk, planes), block 256.  Each block reduces a band of rows.
__global__ void __launch_bounds__(256) stats_partial(const float *__restrict__ f, int H, int W, int pitch,
                                                     int rows_per_block, StatPartial *__restrict__ part)
{
    const int plane = blockIdx.y;
    const int r0 = blockIdx.x * rows_per_block;
    const int r1 = min(H, r0 + rows_per_block);
    float mn = INFINITY, mx = -INFINITY;
    double sum = 0.0;
    int bad = 0;
    const bool vec = ((pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(f) & 15) == 0);
    for (int r = r0; r < r1; ++r) {
        const float *row = f + ((size_t)plane * H + r) * pitch;
        float s = 0.f;  // FP32 partial over one row's share (<= W/256*... values of <= 255-ish)
        if (vec) {
            const int W4 = W >> 2;
            for (int i = threadIdx.x; i < W4; i += blockDim.x) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(row) + i);
                const float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (!isfinite(a[t])) { ++bad; continue; }
                    s += a[t];
                    mn = fminf(mn, a[t]);
                    mx = fmaxf(mx, a[t]);
                }
            }
            for (int x = (W4 << 2) + threadIdx.x; x < W; x += blockDim.x) {
                const float a = __ldg(row + x);
                if (!isfinite(a)) { ++bad; continue; }
                s += a;
                mn = fminf(mn, a);
                mx = fmaxf(mx, a);
            }
        } else {
            for (int x = threadIdx.x; x < W; x += blockDim.x) {
                const float a = __ldg(row + x);
                if (!isfinite(a)) { ++bad; continue; }
                s += a;
                mn = fminf(mn, a);
                mx = fmaxf(mx, a);
            }
        }
        sum += (double)s;
    }
    // block reduction
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
        part[(size_t)plane * gridDim.x + blockIdx.x] = p;
    }
}

// One block.  Reduces the partials of every plane (FP64) and writes PlaneParams.
__global__ void __launch_bounds__(256) stats_finalize(const StatPartial *__restrict__ part, int nblk, int planes,
                                                      long long npix, int centre_given, double tc_given,
                                                      double sigma_r, int K, PlaneParams *__restrict__ pp,
                                                      uint32_t *__restrict__ status)
{
    __shared__ double ssum[256];
    __shared__ float smn[256], smx[256];
    __shared__ int sbad[256];
    uint32_t bits = 0;
    for (int c = 0; c < planes; ++c) {
        double sum = 0.0;
        float mn = INFINITY, mx = -INFINITY;
        int bad = 0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
            const StatPartial p = part[(size_t)c * nblk + b];
            sum += p.sum;
            mn = fminf(mn, p.mn);
            mx = fmaxf(mx, p.mx);
            bad += p.nonfinite;
        }
        ssum[threadIdx.x] = sum;
        smn[threadIdx.x] = mn;
        smx[threadIdx.x] = mx;
        sbad[threadIdx.x] = bad;
        __syncthreads();
        if (threadIdx.x == 0) {
            double S = 0.0;
            float MN = INFINITY, MX = -INFINITY;
            long long BAD = 0;
            for (int t = 0; t < (int)blockDim.x; ++t) {
                S += ssum[t];
                MN = fminf(MN, smn[t]);
                MX = fmaxf(MX, smx[t]);
                BAD += sbad[t];
            }
            PlaneParams q;
            const double mean = S / (double)npix;
            const double tc = centre_given ? tc_given : mean;
            double R = fmax((double)MX - tc, tc - (double)MN);
            int mode = 0;
            if (BAD > 0) {
                mode = 1;
                bits |= 0x2u;
            }
            if (!(R > 0.0)) {
                mode = 1;
                R = 1.0;
            }
            const double s2 = isinf(sigma_r) ? 0.0 : (R / sigma_r) * (R / sigma_r);
            if (mode == 0 && 0.5 * s2 > 80.0) bits |= 0x4u;
            q.tc = (float)tc;
            q.invR = (float)(1.0 / R);
            q.half_s2 = (float)(0.5 * s2);
            q.s2 = (float)s2;
            q.R = (float)R;
            q.mode = mode;
            q.pad0 = q.pad1 = 0;
            q.tc_d = tc;
            q.R_d = R;
            double b = 1.0;
            for (int m = 0; m < KMAX; ++m) {
                if (m == 0) {
                    q.beta[0] = 1.f;
                } else {
                    b = (m == 1) ? 1.0 : b * s2 / (double)m;  // beta_m = s^{2(m-1)} / m!
                    q.beta[m] = (m < K) ? (float)b : 0.f;
                }
            }
            pp[c] = q;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *status = bits;
}

// ------------------------------------------------------------------ row pass

struct RowArgs {
    const float *f;
    float *ws;  // [planes][K][H][Wp]
    const PlaneParams *pp;
    int H, W, pitch, Wp, K, T;  // T: threads per row (power of two, 8..512)
};

// Load one chunk of the row and form u and E (zero beyond the row end).
template <int C>
__device__ __forceinline__ void load_row_chunk(const RowArgs &a, int plane, int row, bool rv, int x0,
                                               const PlaneParams &P, float (&u)[C], float (&phi)[C])
{
    const float *frow = a.f + ((size_t)plane * a.H + (rv ? row : 0)) * a.pitch;
    float v[C];
    const bool vec = ((a.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.f) & 15) == 0) && (x0 + C <= a.W);
    if (rv && vec) {
#pragma unroll
        for (int j = 0; j < C; j += 4) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(frow + x0 + j));
            v[j] = t.x;
            v[j + 1] = t.y;
            v[j + 2] = t.z;
            v[j + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] = (rv && x0 + j < a.W) ? __ldg(frow + x0 + j) : P.tc;
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const bool in = rv && (x0 + j < a.W);
        const float uu = (v[j] - P.tc) * P.invR;
        u[j] = in ? uu : 0.f;
        phi[j] = in ? expf(-P.half_s2 * uu * uu) : 0.f;
    }
}

template <int C>
__device__ __forceinline__ void store_row_chunk(const RowArgs &a, int plane, int k, int row, bool rv, int x0,
                                                const float (&y)[C], float beta)
{
    if (!rv) return;
    float *out = a.ws + (((size_t)plane * a.K + k) * a.H + row) * a.Wp;
    if (x0 + C <= a.Wp) {
#pragma unroll
        for (int j = 0; j < C; j += 4)
            *reinterpret_cast<float4 *>(out + x0 + j) =
                make_float4(y[j] * beta, y[j + 1] * beta, y[j + 2] * beta, y[j + 3] * beta);
    } else {
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (x0 + j < a.Wp) out[x0 + j] = y[j] * beta;
    }
}

// grid (ceil(H / rows_per_cta), planes); block = max(T, 256) threads.
template <int C>
__global__ void __launch_bounds__(512) row_iir(RowArgs a, IIRCoef cf)
{
    // cross-warp totals: [parity][slot = r_local * wpr + warp_in_row][pole] (cr, ci, ar, ai)
    __shared__ float4 tot[2][16][NP];
    const int T = a.T;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int plane = blockIdx.y;
    const int rows_per_cta = blockDim.x / T;
    const int r_local = tid / T;
    const int t = tid % T;
    const int row = blockIdx.x * rows_per_cta + r_local;
    const bool rv = row < a.H;
    const PlaneParams &P = a.pp[plane];
    const int L = T < 32 ? T : 32;  // segment width inside a warp
    const int ls = lane & (L - 1);
    const int wpr = T >> 5;         // warps per row (0 if T < 32)
    const int wr = t >> 5;          // warp index inside the row
    const int x0 = t * C;
    const int mode = P.mode;

    float u[C], phi[C];
    load_row_chunk<C>(a, plane, row, rv, x0, P, u, phi);

    if (mode != 0) {
        // copy mode: the column pass copies f; nothing to filter.
        return;
    }

    // per-thread powers for the cross-warp carries: p^{C ls} and p^{C (31 - ls)}
    float qcr[NP], qci[NP], qar[NP], qai[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        cpow_tab(qcr[m], qci[m], cf, m, ls);
        cpow_tab(qar[m], qai[m], cf, m, 31 - ls);
    }

#pragma unroll 1
    for (int k = 0; k < a.K; ++k) {
        if (k > 0) {
#pragma unroll
            for (int j = 0; j < C; ++j) phi[j] *= u[j];
        }
        float y[C];
        float er[NP], ei[NP], sr[NP], si[NP];
        chunk_local<C>(phi, y, er, ei, sr, si, cf);

        // segment scan across the T chunks of the row
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
        if (wpr > 1) {
            const int par = k & 1;
            const int slot = r_local * wpr + wr;
            if (lane == 31) {
#pragma unroll
                for (int m = 0; m < NP; ++m) {
                    tot[par][slot][m].x = er[m];
                    tot[par][slot][m].y = ei[m];
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int m = 0; m < NP; ++m) {
                    tot[par][slot][m].z = sr[m];
                    tot[par][slot][m].w = si[m];
                }
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                // P^32 = table index 5
                const float p32r = cf.Pr[m][5], p32i = cf.Pi[m][5];
                float Cr = 0.f, Ci = 0.f;
                for (int w = 0; w < wr; ++w) {
                    const float4 tt = tot[par][r_local * wpr + w][m];
                    float nr, ni;
                    cmul(nr, ni, p32r, p32i, Cr, Ci);
                    Cr = nr + tt.x;
                    Ci = ni + tt.y;
                }
                float Ar = 0.f, Ai = 0.f;
                for (int w = wpr - 1; w > wr; --w) {
                    const float4 tt = tot[par][r_local * wpr + w][m];
                    float nr, ni;
                    cmul(nr, ni, p32r, p32i, Ar, Ai);
                    Ar = nr + tt.z;
                    Ai = ni + tt.w;
                }
                cmadd(cr[m], ci[m], qcr[m], qci[m], Cr, Ci);
                cmadd(ar[m], ai[m], qar[m], qai[m], Ar, Ai);
            }
        }
        chunk_correct<C>(y, cr, ci, ar, ai, cf);
        store_row_chunk<C>(a, plane, k, row, rv, x0, y, P.beta[k]);
    }
}

// FIR row pass: the row's channel is staged in shared memory with zero halos.
// grid (ceil(H / rows_per_cta), planes); block = max(T, 256) threads.
template <int C, int WH>
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
    if (P.mode != 0) return;

    float u[C], phi[C];
    load_row_chunk<C>(a, plane, row, rv, x0, P, u, phi);
    // zero both halos of both parity buffers
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
        if (k > 0) {
#pragma unroll
            for (int j = 0; j < C; ++j) phi[j] *= u[j];
        }
        float *buf = srow + ((k & 1) * rows_per_cta + r_local) * span;
#pragma unroll
        for (int j = 0; j < C; ++j) buf[WH + x0 + j] = phi[j];
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
    float *y;
    const PlaneParams *pp;
    uint32_t *status;
    int H, W, pitch, Wp, K, N;
};

// Per-pixel combine state: descending m, d = d u + v; v = v u + Psi_m;
// q = q u + Psi_m for 1 <= m <= N.
template <int C>
__device__ __forceinline__ void combine_step(int m, int N, const float (&u)[C], float (&q)[C], float (&v)[C],
                                             float (&d)[C], const float (&psi)[C])
{
    if (m >= 1 && m <= N) {
#pragma unroll
        for (int j = 0; j < C; ++j) q[j] = fmaf(u[j], q[j], psi[j]);
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
        d[j] = fmaf(u[j], d[j], v[j]);
        v[j] = fmaf(u[j], v[j], psi[j]);
    }
}

__device__ __forceinline__ float finish_pixel(const PlaneParams &P, float f, float u, float q, float d, float psi0,
                                              bool &nonpos)
{
    if (P.mode != 0) return f;
    const float Q = fmaf(P.s2 * u, q, psi0);
    if (!(Q > 0.f)) {
        nonpos = true;
        return __int_as_float(0x7fc00000);
    }
    return fmaf(P.R, __fdiv_rn(d, Q), P.tc);
}

// Column pass for the recursive filter.  A cluster of CL CTAs covers the
// full height of an 8-column strip; CTA rank r owns rows [r*32*C, (r+1)*32*C).
// Thread (warp w, lane l): column l%8 of the strip, chunk 4w + l/8 of the CTA.
// grid (strips * CL, planes), block 256, cluster (CL, 1, 1).
template <int C, bool CLUSTER>
__global__ void __launch_bounds__(256, 2) col_iir(ColArgs a, IIRCoef cf)
{
    __shared__ float4 wt[2][8][8][NP];  // [parity][warp][col][pole] (causal total, anticausal total)
    __shared__ float4 ct[2][8][NP];     // [parity][col][pole] CTA totals
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int col = lane & 7, l4 = lane >> 3;
    const int plane = blockIdx.y;
    int rank = 0, CL = 1;
    if (CLUSTER) {
        cg::cluster_group cl = cg::this_cluster();
        rank = (int)cl.block_rank();
        CL = (int)cl.num_blocks();
    }
    const int strip = blockIdx.x / CL;
    const int x = strip * 8 + col;
    const int chunk_cta = warp * 4 + l4;
    const int row0 = (rank * 32 + chunk_cta) * C;
    const PlaneParams &P = a.pp[plane];

    // input pixels of the chunk (for u) and the combine state
    float u[C], q[C], v[C], d[C];
    const float *fcol = a.f + (size_t)plane * a.H * a.pitch;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int r = row0 + j;
        const bool in = (r < a.H) && (x < a.W);
        const float fv = in ? __ldg(fcol + (size_t)r * a.pitch + x) : 0.f;
        u[j] = (fv - P.tc) * P.invR;
        q[j] = v[j] = d[j] = 0.f;
    }
    const bool filt = (P.mode == 0);

    // per-thread powers p^{C l4}, p^{C (3 - l4)} and, for the cluster carry,
    // p^{C 4 warp}, p^{C 4 (7 - warp)}
    float qcr[NP], qci[NP], qar[NP], qai[NP];
    float wcr[NP], wci[NP], war[NP], wai[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        cpow_tab(qcr[m], qci[m], cf, m, l4);
        cpow_tab(qar[m], qai[m], cf, m, 3 - l4);
        if (CLUSTER) {
            cpow_tab(wcr[m], wci[m], cf, m, 4 * warp);
            cpow_tab(war[m], wai[m], cf, m, 4 * (7 - warp));
        }
    }

    float psi0[C];
    const float *wsp = a.ws + (size_t)plane * a.K * a.H * a.Wp;
#pragma unroll 1
    for (int k = a.K - 1; k >= 0; --k) {
        float xin[C];
        const float *src = wsp + (size_t)k * a.H * a.Wp + x;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const int r = row0 + j;
            xin[j] = (filt && r < a.H) ? __ldg(src + (size_t)r * a.Wp) : 0.f;
        }
        float y[C];
        float er[NP], ei[NP], sr[NP], si[NP];
        chunk_local<C>(xin, y, er, ei, sr, si, cf);

        // level 1: the 4 chunks of this column inside the warp (lane stride 8)
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
        // level 2: the 8 warps of the CTA
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
        __syncthreads();
        float Cwr[NP], Cwi[NP], Awr[NP], Awi[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float p4r = cf.Pr[m][2], p4i = cf.Pi[m][2];
            float Cr = 0.f, Ci = 0.f;
            for (int w = 0; w < warp; ++w) {
                const float4 tt = wt[par][w][col][m];
                float nr, ni;
                cmul(nr, ni, p4r, p4i, Cr, Ci);
                Cr = nr + tt.x;
                Ci = ni + tt.y;
            }
            float Ar = 0.f, Ai = 0.f;
            for (int w = 7; w > warp; --w) {
                const float4 tt = wt[par][w][col][m];
                float nr, ni;
                cmul(nr, ni, p4r, p4i, Ar, Ai);
                Ar = nr + tt.z;
                Ai = ni + tt.w;
            }
            Cwr[m] = Cr;
            Cwi[m] = Ci;
            Awr[m] = Ar;
            Awi[m] = Ai;
        }
        if (CLUSTER) {
            // CTA totals: causal from warp 7 (its l4 == 3 lanes), anticausal from warp 0 (l4 == 0)
            if (warp == 7 && l4 == 3) {
#pragma unroll
                for (int m = 0; m < NP; ++m) {
                    float tr = er[m], ti = ei[m];
                    cmadd(tr, ti, cf.Pr[m][2], cf.Pi[m][2], Cwr[m], Cwi[m]);
                    ct[par][col][m].x = tr;
                    ct[par][col][m].y = ti;
                }
            }
            if (warp == 0 && l4 == 0) {
#pragma unroll
                for (int m = 0; m < NP; ++m) {
                    float tr = sr[m], ti = si[m];
                    cmadd(tr, ti, cf.Pr[m][2], cf.Pi[m][2], Awr[m], Awi[m]);
                    ct[par][col][m].z = tr;
                    ct[par][col][m].w = ti;
                }
            }
            cg::cluster_group cl = cg::this_cluster();
            cl.sync();
            // level 3: CTAs of the cluster (P^32 = table index 5)
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const float p32r = cf.Pr[m][5], p32i = cf.Pi[m][5];
                float Cr = 0.f, Ci = 0.f;
                for (int r = 0; r < rank; ++r) {
                    const float4 *rem = cl.map_shared_rank(&ct[par][col][m], r);
                    const float4 tt = *rem;
                    float nr, ni;
                    cmul(nr, ni, p32r, p32i, Cr, Ci);
                    Cr = nr + tt.x;
                    Ci = ni + tt.y;
                }
                float Ar = 0.f, Ai = 0.f;
                for (int r = CL - 1; r > rank; --r) {
                    const float4 *rem = cl.map_shared_rank(&ct[par][col][m], r);
                    const float4 tt = *rem;
                    float nr, ni;
                    cmul(nr, ni, p32r, p32i, Ar, Ai);
                    Ar = nr + tt.z;
                    Ai = ni + tt.w;
                }
                // propagate the CTA carry through the 4*warp chunks before this warp
                cmadd(Cwr[m], Cwi[m], wcr[m], wci[m], Cr, Ci);
                cmadd(Awr[m], Awi[m], war[m], wai[m], Ar, Ai);
            }
        }
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            cmadd(cr[m], ci[m], qcr[m], qci[m], Cwr[m], Cwi[m]);
            cmadd(ar[m], ai[m], qar[m], qai[m], Awr[m], Awi[m]);
        }
        chunk_correct<C>(y, cr, ci, ar, ai, cf);
        if (k == 0) {
#pragma unroll
            for (int j = 0; j < C; ++j) psi0[j] = y[j];
            // P~ needs the final derivative step only
#pragma unroll
            for (int j = 0; j < C; ++j) d[j] = fmaf(u[j], d[j], v[j]);
        } else {
            combine_step<C>(k, a.N, u, q, v, d, y);
        }
    }
    if (CLUSTER) {
        // no CTA may leave while a peer can still read its shared memory
        cg::this_cluster().sync();
    }
    bool nonpos = false;
    float *ycol = a.y + (size_t)plane * a.H * a.pitch;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const int r = row0 + j;
        if (r < a.H && x < a.W) {
            const float fv = filt ? 0.f : __ldg(fcol + (size_t)r * a.pitch + x);
            ycol[(size_t)r * a.pitch + x] = finish_pixel(P, fv, u[j], q[j], d[j], psi0[j], nonpos);
        }
    }
    if (__any_sync(0xffffffffu, nonpos) && lane == 0) atomicOr(a.status, 0x1u);
}

// Column pass for the FIR filter: 2-D tiles of 32 columns x 64 rows; the
// channel's tile plus a WH-row halo is staged in shared memory.
// grid (ceil(W/32), ceil(H/64), planes), block 256 (32 columns x 8 row groups of 8).
template <int WH>
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
    float u[RPT], q[RPT], v[RPT], d[RPT], fv[RPT], psi0[RPT];
    const float *fp = a.f + (size_t)plane * a.H * a.pitch;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = rbase + ty * RPT + j;
        const bool in = (r < a.H) && (x < a.W);
        fv[j] = in ? __ldg(fp + (size_t)r * a.pitch + x) : 0.f;
        u[j] = (fv[j] - P.tc) * P.invR;
        q[j] = v[j] = d[j] = psi0[j] = 0.f;
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
            if (k == 0) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    psi0[j] = y[j];
                    d[j] = fmaf(u[j], d[j], v[j]);
                }
            } else {
                combine_step<RPT>(k, a.N, u, q, v, d, y);
            }
        }
    }
    bool nonpos = false;
    float *yp = a.y + (size_t)plane * a.H * a.pitch;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = rbase + ty * RPT + j;
        if (r < a.H && x < a.W) yp[(size_t)r * a.pitch + x] = finish_pixel(P, fv[j], u[j], q[j], d[j], psi0[j], nonpos);
    }
    if (__any_sync(0xffffffffu, nonpos) && tx == 0) atomicOr(a.status, 0x1u);
}

}  // namespace bfgp
