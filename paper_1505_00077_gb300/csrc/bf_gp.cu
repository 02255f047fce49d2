// bf_gp.cu -- host side of the C ABI declared in include/bf_gp.h.
//
// Validates arguments, lays out the caller's workspace, derives the spatial
// filter coefficients in FP64 (rounded once to FP32) and enqueues the kernels
// of bf_gp_device.cuh on the caller's stream.  Never allocates device memory.
#include <cmath>
#include <complex>
#include <cstdio>
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/bf_gp.h"
#include "bf_gp_device.cuh"

using namespace bfgp;

namespace {

thread_local char g_cuda_err[256] = "";

bf_status cuda_fail(cudaError_t e, const char *where)
{
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", where, cudaGetErrorString(e));
    return BF_ERR_CUDA;
}

#define BF_CUDA(call)                                    \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr int ROW_C = 16;           // samples per thread along a row
constexpr int COL_C = 16;           // rows per thread along a column
constexpr int COL_ROWS_PER_CTA = COL_ROWS;  // 32 chunks of COL_C rows
constexpr int COL_MAX_CLUSTER_TC = 8;  // column cluster limit of the tensor-core column passes
constexpr size_t HDR_BYTES = 4096;  // status word + spare

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

struct Plan {
    int K, N, Wp, w, spatial;  // spatial: 1 FIR, 2 IIR
    int nblk, rows_per_block;
    int T;                     // row threads per row
    int CL;                    // column cluster size (IIR)
    int row_tc, col_tc;        // recursive filter: row / column pass engine (0 CUDA cores, 1 mma.sync, 2 tcgen05)
    int row_block;             // threads per CTA of the row pass asked for (0 = default)
    int fir_tile;              // fused FIR: output tile height (16, 32 or 64 rows)
    int engine_auto;           // opts.engine == 0 (the adjoint row pass then runs on CUDA cores)
    int joint;                 // joint filter: K = 2 (N + 1), CUDA-core passes
    int box_passes, box_r;     // box variant: passes of a flat kernel of half-width box_r (w = passes * box_r)
    int wpr;                   // tensor-core row pass: warps per row (512 samples each)
    size_t off_params, off_part, off_acc, off_planes, total;
};

int fir_halfwidth(float sigma_s, const bf_gp_opts *o)
{
    if (o->fir_halfwidth > 0) return o->fir_halfwidth;
    return (int)std::ceil(3.0 * (double)sigma_s - 1e-12);
}

bf_status check_opts(const bf_gp_opts *o)
{
    if (o->order < 0 || o->order > KMAX - 2) return BF_ERR_INVALID_ARG;
    if (o->spatial < 0 || o->spatial > 3) return BF_ERR_INVALID_ARG;
    if (o->centre < 0 || o->centre > 1) return BF_ERR_INVALID_ARG;
    if (o->fir_halfwidth < 0) return BF_ERR_INVALID_ARG;
    if (o->centre == BF_CENTRE_GIVEN && !std::isfinite(o->t_c)) return BF_ERR_INVALID_ARG;
    if (o->engine < 0 || o->engine > 3) return BF_ERR_INVALID_ARG;
    if (o->fir_two_pass < 0 || o->fir_two_pass > 1) return BF_ERR_INVALID_ARG;
    if (o->box_passes < 0 || o->box_passes > 3) return BF_ERR_INVALID_ARG;
    if (o->tc5_wait_test < 0) return BF_ERR_INVALID_ARG;
    if (o->row_threads != 0 && o->row_threads != 256 && o->row_threads != 512) return BF_ERR_INVALID_ARG;
    if (o->fir_tile != 0 && o->fir_tile != 16 && o->fir_tile != 32 && o->fir_tile != 64) return BF_ERR_INVALID_ARG;
    for (int i = 0; i < 2; ++i)
        if (o->reserved[i] != 0) return BF_ERR_INVALID_ARG;
    return BF_OK;
}

bf_status make_plan(int planes, int H, int W, float sigma_s, const bf_gp_opts *o, Plan *p, int joint = 0)
{
    if (planes < 1 || H < 1 || W < 1) return BF_ERR_INVALID_ARG;
    if (!(sigma_s > 0.f) || !std::isfinite(sigma_s)) return BF_ERR_INVALID_ARG;
    bf_status st = check_opts(o);
    if (st != BF_OK) return st;
    if (joint && 2 * (o->order + 1) > KMAX) return BF_ERR_INVALID_ARG;
    p->joint = joint;
    p->N = o->order;
    p->K = joint ? 2 * (o->order + 1) : o->order + 2;
    p->w = fir_halfwidth(sigma_s, o);
    int sp = o->spatial;
    p->box_passes = 0;
    p->box_r = 0;
    if (sp == BF_SPATIAL_BOX) {
        // box variant: passes x half-width r; the window the fused kernel stages is passes * r
        const int P = o->box_passes ? o->box_passes : 3;
        int r = o->fir_halfwidth;
        if (r <= 0) {
            const double s2 = (double)sigma_s * (double)sigma_s;
            r = (int)std::lround((std::sqrt(12.0 * s2 / P + 1.0) - 1.0) / 2.0);
            if (r < 1) r = 1;
        }
        if (P * r > FIR_WMAX || joint) return BF_ERR_UNSUPPORTED;
        p->box_passes = P;
        p->box_r = r;
        p->w = P * r;
    }
    if (sp == BF_SPATIAL_AUTO) sp = (p->w <= FIR_WMAX) ? BF_SPATIAL_FIR : BF_SPATIAL_IIR;
    if (sp == BF_SPATIAL_FIR && p->w > FIR_WMAX) return BF_ERR_UNSUPPORTED;
    p->spatial = sp;
    p->Wp = (int)align_up((size_t)W, 32);
    p->T = next_pow2((W + ROW_C - 1) / ROW_C);
    if (p->T < 8) p->T = 8;
    if (p->T > 512) return BF_ERR_UNSUPPORTED;  // rows longer than 8192 samples
    p->CL = (H + COL_ROWS_PER_CTA - 1) / COL_ROWS_PER_CTA;
    p->row_tc = (!joint && (o->engine == 0 || o->engine == 2)) ? 1 : 0;
    p->engine_auto = o->engine == 0 ? 1 : 0;
    p->col_tc = joint ? 0 : (o->engine == 2 ? 1 : (o->engine == 3 ? 2 : 0));
    p->wpr = next_pow2((W + 511) / 512);
    p->row_block = o->row_threads;
    p->fir_tile = o->fir_tile ? o->fir_tile : 32;
    if (sp == BF_SPATIAL_IIR && p->row_tc && p->wpr > 16) return BF_ERR_UNSUPPORTED;
    // columns longer than 8192 (CUDA-core column pass) or 4096 (tensor-core column passes)
    if (sp == BF_SPATIAL_IIR && p->CL > (p->col_tc ? COL_MAX_CLUSTER_TC : COL_MAX_CTAS)) return BF_ERR_UNSUPPORTED;
    const long long px = (long long)H * W;
    // stats partials: at most 1024 blocks, at least 2048 pixels each (small images still spread
    // over many SMs; every block's loads are independent)
    const long long per_blk = std::max<long long>(2048, (px + 1023) / 1024);
    int nblk = (int)std::min<long long>((long long)H, std::max<long long>(1, (px + per_blk - 1) / per_blk));
    p->rows_per_block = (H + nblk - 1) / nblk;
    p->nblk = (H + p->rows_per_block - 1) / p->rows_per_block;
    size_t off = HDR_BYTES;
    p->off_params = off;
    off = align_up(off + sizeof(PlaneParams) * (size_t)planes, 256);
    p->off_part = off;
    off = align_up(off + sizeof(StatPartial) * (size_t)planes * p->nblk, 256);
    p->off_acc = off;
    off = align_up(off + sizeof(double) * NACC * (size_t)planes, 256);
    p->off_planes = off;
    off = align_up(off + sizeof(float) * (size_t)planes * p->K * H * p->Wp, 256);
    p->total = off;
    return BF_OK;
}

void deriche_coefs(double sigma, int C, IIRCoef *cf)
{
    // Deriche's published 4th-order fit of exp(-x^2/2) (unit scale):
    //   (a0 cos(w0 x) + a1 sin(w0 x)) e^{-b0 x} + (c0 cos(w1 x) + c1 sin(w1 x)) e^{-b1 x},
    // i.e. Re[A0 p0^d + A1 p1^d] at x = d/sigma with p = exp((-b + i w)/sigma).
    const double a0 = 1.680, a1 = 3.735, b0 = 1.783, b1 = 1.723;
    const double c0 = -0.6803, c1 = -0.2598, w0 = 0.6318, w1 = 1.997;
    const std::complex<double> p[NP] = {std::exp(std::complex<double>(-b0, w0) / sigma),
                                        std::exp(std::complex<double>(-b1, w1) / sigma)};
    const std::complex<double> A[NP] = {{a0, -a1}, {c0, -c1}};
    std::memset(cf, 0, sizeof *cf);
    for (int m = 0; m < NP; ++m) {
        cf->pr[m] = (float)p[m].real();
        cf->pi[m] = (float)p[m].imag();
        for (int e = 0; e <= C; ++e) {
            const std::complex<double> t = A[m] * std::pow(p[m], (double)e);
            cf->tr[m][e] = (float)t.real();
            cf->ti[m][e] = (float)t.imag();
        }
        for (int i = 0; i < 12; ++i) {
            const std::complex<double> t = std::pow(p[m], (double)C * (double)(1 << i));
            cf->Pr[m][i] = (float)t.real();
            cf->Pi[m][i] = (float)t.imag();
        }
        for (int e = 0; e <= 8; ++e) {
            const std::complex<double> t = std::pow(p[m], (double)e);
            cf->wr[m][e] = (float)t.real();
            cf->wi[m][e] = (float)t.imag();
        }
    }
    for (int d = 0; d < 8; ++d) {
        double h = 0.0;
        for (int m = 0; m < NP; ++m) h += (A[m] * std::pow(p[m], (double)d)).real();
        cf->h[d] = (float)h;
    }
    // pairs for the two-lane FMA: the same FP32 values
    for (int m = 0; m < NP; ++m) {
        for (int i = 0; i < 8; ++i) {
            cf->wc[m][i] = make_float2(cf->wr[m][7 - i], cf->wi[m][7 - i]);
            cf->wa[m][i] = make_float2(cf->wr[m][i], cf->wi[m][i]);
        }
        for (int j = 0; j < 8; j += 2) {
            cf->kc[m][j >> 1] = make_float2(cf->tr[m][j + 1], cf->tr[m][j + 2]);
            cf->kcn[m][j >> 1] = make_float2(-cf->ti[m][j + 1], -cf->ti[m][j + 2]);
            cf->ka[m][j >> 1] = make_float2(cf->tr[m][8 - j], cf->tr[m][7 - j]);
            cf->kan[m][j >> 1] = make_float2(-cf->ti[m][8 - j], -cf->ti[m][7 - j]);
        }
    }
    for (int d = -7; d <= 7; ++d) cf->hp[d + 7] = make_float2(cf->h[std::abs(d)], cf->h[std::abs(d + 1) < 8 ? std::abs(d + 1) : 7]);
}

// The three 8 x 8 matrices of the tensor-core passes (chunk length 8), FP64 -> FP32:
//   loc[k][n] = h(|n - k|);  sum[k][2c + ri]: chunk end states of combo c (c = 0, 1 causal pole c:
//   p^{7-k}; c = 2, 3 anticausal pole c - 2: p^k), ri = 0 real, 1 imaginary part;
//   cor[c][n] = Re(B), cor[c + 4][n] = -Im(B) with B = A p^{n+1} (causal) or A p^{8-n} (anticausal).
void tc_mats(double sigma, TCMat *tm)
{
    const double a0 = 1.680, a1 = 3.735, b0 = 1.783, b1 = 1.723;
    const double c0 = -0.6803, c1 = -0.2598, w0 = 0.6318, w1 = 1.997;
    const std::complex<double> p[NP] = {std::exp(std::complex<double>(-b0, w0) / sigma),
                                        std::exp(std::complex<double>(-b1, w1) / sigma)};
    const std::complex<double> A[NP] = {{a0, -a1}, {c0, -c1}};
    std::memset(tm, 0, sizeof *tm);
    for (int k = 0; k < 8; ++k)
        for (int n = 0; n < 8; ++n) {
            double h = 0.0;
            for (int m = 0; m < NP; ++m) h += (A[m] * std::pow(p[m], (double)std::abs(n - k))).real();
            tm->loc[k][n] = (float)h;
        }
    for (int k = 0; k < 8; ++k)
        for (int c = 0; c < 4; ++c) {
            const int m = c & 1;
            const std::complex<double> v = c < 2 ? std::pow(p[m], (double)(7 - k)) : std::pow(p[m], (double)k);
            tm->sum[k][2 * c] = (float)v.real();
            tm->sum[k][2 * c + 1] = (float)v.imag();
        }
    for (int c = 0; c < 4; ++c) {
        const int m = c & 1;
        for (int n = 0; n < 8; ++n) {
            const std::complex<double> B = c < 2 ? A[m] * std::pow(p[m], (double)(n + 1)) : A[m] * std::pow(p[m], (double)(8 - n));
            tm->cor[c][n] = (float)B.real();
            tm->cor[c + 4][n] = (float)(-B.imag());
        }
    }
}

void fir_coefs(double sigma, int w, FIRCoef *g)
{
    std::memset(g, 0, sizeof *g);
    for (int d = 0; d <= w && d <= FIR_WMAX; ++d) g->g[d] = (float)std::exp(-(double)d * d / (2.0 * sigma * sigma));
}

// ---------------------------------------------------------------- launches

template <int WH, int MODE>
bf_status launch_row_fir_w(const RowArgs &ra, const FIRCoef &g, int planes, cudaStream_t s, int row_block)
{
    const int T = ra.T;
    const int want = row_block ? row_block : 256;
    const int block = T > want ? T : want;
    const int rows_per_cta = block / T;
    const size_t smem = sizeof(float) * 2 * rows_per_cta * (size_t)(T * ROW_C + 2 * WH);
    BF_CUDA(cudaFuncSetAttribute(row_fir<ROW_C, WH, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((ra.H + rows_per_cta - 1) / rows_per_cta, planes);
    row_fir<ROW_C, WH, MODE><<<grid, block, smem, s>>>(ra, g);
    return BF_OK;
}

template <int WH, int MODE>
bf_status launch_col_fir_w(const ColArgs &ca, const FIRCoef &g, int planes, cudaStream_t s)
{
    dim3 grid((ca.W + 31) / 32, (ca.H + 63) / 64, planes);
    col_fir<WH, MODE><<<grid, 256, 0, s>>>(ca, g);
    return BF_OK;
}

}  // namespace

namespace {

struct Call {
    Plan p;
    cudaStream_t s;
    uint32_t *status;
    PlaneParams *pp;
    StatPartial *part;
    double *acc;
    float *planesbuf;
    RowArgs ra;
    ColArgs ca;
};

// Validates the common arguments and lays out the workspace.  out: y for the
// forward, grad_f for the backward (may be null for the stats/rows phases).
bf_status prepare(const float *f, float *out, int planes, int H, int W, int pitch, float sigma_s, float sigma_r,
                  const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream, bool need_out, Call *c,
                  const float *data = nullptr)
{
    if (!f || !ws || (need_out && !out)) return BF_ERR_INVALID_ARG;
    if (pitch < W) return BF_ERR_INVALID_ARG;
    if (!(sigma_r > 0.f)) return BF_ERR_INVALID_ARG;  // also rejects NaN; +inf accepted
    // the kernels load and store whole floats
    for (const void *p : {(const void *)f, (const void *)out, (const void *)data})
        if ((reinterpret_cast<uintptr_t>(p) & 3) != 0) return BF_ERR_INVALID_ARG;
    bf_gp_opts d;
    if (!opts) {
        bf_gp_default_opts(&d);
        opts = &d;
    }
    bf_status st = make_plan(planes, H, W, sigma_s, opts, &c->p, data ? 1 : 0);
    if (st != BF_OK) return st;
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < c->p.total) return BF_ERR_WORKSPACE;
    if (need_out) {
        // inputs and output must not overlap
        const char *yb = reinterpret_cast<const char *>(out);
        const size_t span = sizeof(float) * ((size_t)planes * H * pitch);
        for (const float *in : {f, data}) {
            if (!in) continue;
            const char *fb = reinterpret_cast<const char *>(in);
            if (fb < yb + span && yb < fb + span) return BF_ERR_INVALID_ARG;
        }
    }
    c->s = reinterpret_cast<cudaStream_t>(stream);
    char *wsb = static_cast<char *>(ws);
    c->status = reinterpret_cast<uint32_t *>(wsb);
    c->pp = reinterpret_cast<PlaneParams *>(wsb + c->p.off_params);
    c->part = reinterpret_cast<StatPartial *>(wsb + c->p.off_part);
    c->acc = reinterpret_cast<double *>(wsb + c->p.off_acc);
    c->planesbuf = reinterpret_cast<float *>(wsb + c->p.off_planes);
    RowArgs &ra = c->ra;
    std::memset(&ra, 0, sizeof ra);
    ra.f = f;
    ra.fd = data;
    ra.ws = c->planesbuf;
    ra.pp = c->pp;
    ra.acc = c->acc;
    ra.H = H;
    ra.W = W;
    ra.pitch = pitch;
    ra.Wp = c->p.Wp;
    ra.K = c->p.K;
    ra.T = c->p.T;
    ra.N = c->p.N;
    ColArgs &ca = c->ca;
    std::memset(&ca, 0, sizeof ca);
    ca.ws = c->planesbuf;
    ca.f = f;
    ca.gy = data;  // joint filter: the data image (copied for planes the filter does not run on)
    ca.y = out;
    ca.pp = c->pp;
    ca.status = c->status;
    ca.acc = c->acc;
    ca.H = H;
    ca.W = W;
    ca.pitch = pitch;
    ca.Wp = c->p.Wp;
    ca.K = c->p.K;
    ca.N = c->p.N;
    ca.wait_limit = opts->tc5_wait_test > 0 ? opts->tc5_wait_test : MBAR_LIMIT;
    ca.no_mma = opts->tc5_wait_test > 0 ? 1 : 0;
    return BF_OK;
}

// src / copy: when given, the statistics pass reads the input from src
// (mapped host memory) and stores it into copy, the device input of the call.
bf_status run_stats(const Call &c, int planes, int H, int W, int pitch, float sigma_s, float sigma_r,
                    const bf_gp_opts *opts, int for_backward, const float *src = nullptr, float *copy = nullptr)
{
    bf_gp_opts d;
    if (!opts) {
        bf_gp_default_opts(&d);
        opts = &d;
    }
    if (src)
        stats_partial<true><<<dim3(c.p.nblk, planes), 256, 0, c.s>>>(src, H, W, pitch, c.p.rows_per_block, c.part,
                                                                     c.status, copy);
    else
        stats_partial<false><<<dim3(c.p.nblk, planes), 256, 0, c.s>>>(c.ra.f, H, W, pitch, c.p.rows_per_block,
                                                                      c.part, c.status, nullptr);
    stats_finalize<<<planes, 256, 0, c.s>>>(c.part, c.p.nblk, (long long)H * W,
                                            opts->centre == BF_CENTRE_GIVEN ? 1 : 0, opts->t_c, (double)sigma_r,
                                            (double)sigma_s, c.p.K, for_backward, c.pp, c.status);
    BF_CUDA(cudaGetLastError());
    return BF_OK;
}

template <int MODE>
bf_status run_rows(const Call &c, int planes, float sigma_s)
{
    if (c.p.spatial == BF_SPATIAL_BOX) return BF_ERR_UNSUPPORTED;  // the box variant runs fused only
    const int T = c.ra.T;
    const int want = c.p.row_block ? c.p.row_block : 256;  // threads per CTA asked for
    const int block = T > want ? T : want;
    const int rows_per_cta = block / T;
    if (c.p.spatial == BF_SPATIAL_FIR) {
        FIRCoef g;
        fir_coefs((double)sigma_s, c.p.w, &g);
        bf_status st = BF_ERR_UNSUPPORTED;
        switch (c.p.w) {
#define BF_CASE(WW) \
    case WW: st = launch_row_fir_w<WW, MODE>(c.ra, g, planes, c.s, c.p.row_block); break;
            BF_CASE(1) BF_CASE(2) BF_CASE(3) BF_CASE(4) BF_CASE(5) BF_CASE(6)
            BF_CASE(7) BF_CASE(8) BF_CASE(9) BF_CASE(10) BF_CASE(11) BF_CASE(12)
#undef BF_CASE
        default: break;
        }
        if (st != BF_OK) return st;
    } else if (c.p.row_tc && !(MODE == MODE_ADJ && c.p.engine_auto)) {
        // (engine auto runs the adjoint row pass on CUDA cores: measured faster for it at every size)
        IIRCoef cr;
        deriche_coefs((double)sigma_s, TC_C, &cr);
        TCMat tm;
        tc_mats((double)sigma_s, &tm);
        RowArgs ra = c.ra;
        ra.T = c.p.wpr;  // warps per row
        const int tblock = 32 * c.p.wpr > want ? 32 * c.p.wpr : want;
        const int trows = (tblock / 32) / c.p.wpr;
        dim3 grid((c.ra.H + trows - 1) / trows, planes);
        if constexpr (MODE != MODE_JOINT) row_tc<MODE><<<grid, tblock, 0, c.s>>>(ra, cr, tm);
    } else {
        IIRCoef cr;
        deriche_coefs((double)sigma_s, ROW_C, &cr);
        dim3 grid((c.ra.H + rows_per_cta - 1) / rows_per_cta, planes);
        row_iir<ROW_C, MODE><<<grid, block, 0, c.s>>>(c.ra, cr);
    }
    BF_CUDA(cudaGetLastError());
    return BF_OK;
}

// B operand of the tcgen05 half-chunk products (FP64 -> FP32, then TF32 high
// part with round-to-nearest-away and the FP32 remainder), in the K-major
// core-matrix layout: (n, i) at float (n/8)*64 + (i/4)*32 + (n%8)*4 + i%4.
//   n = 0..7: h(|n - i|);  n = 8 + 2m (+1): Re (Im) p_m^{7-i};  n = 12 + 2m (+1): Re (Im) p_m^i
float tf32_rna(float v)
{
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

void umma_mats(double sigma, UMat *um)
{
    const double a0 = 1.680, a1 = 3.735, b0 = 1.783, b1 = 1.723;
    const double c0 = -0.6803, c1 = -0.2598, w0 = 0.6318, w1 = 1.997;
    const std::complex<double> p[NP] = {std::exp(std::complex<double>(-b0, w0) / sigma),
                                        std::exp(std::complex<double>(-b1, w1) / sigma)};
    const std::complex<double> A[NP] = {{a0, -a1}, {c0, -c1}};
    std::memset(um, 0, sizeof *um);
    for (int n = 0; n < 16; ++n)
        for (int i = 0; i < 8; ++i) {
            double v;
            if (n < 8) {
                v = 0.0;
                for (int m = 0; m < NP; ++m) v += (A[m] * std::pow(p[m], (double)std::abs(n - i))).real();
            } else {
                const int q = n - 8, m = (q >> 1) & 1, im = q & 1;
                const std::complex<double> t = std::pow(p[m], (double)(q < 4 ? 7 - i : i));
                v = im ? t.imag() : t.real();
            }
            const float f = (float)v;
            const int o = (n / 8) * 64 + (i / 4) * 32 + (n % 8) * 4 + i % 4;
            um->hi[o] = tf32_rna(f);
            um->lo[o] = f - um->hi[o];
        }
}

// The fused FIR kernel with tile height TH (window half-width from the plan).
template <int TH>
bf_status launch_fir_fused(const Call &c, int planes, const FIRCoef &g)
{
    dim3 grid((c.ca.W + 31) / 32, (c.ca.H + TH - 1) / TH, planes);
    switch (c.p.w) {
#define BF_CASE(WW) \
    case WW: fir_fused<WW, 0, TH><<<grid, 256, 0, c.s>>>(c.ca, g); break;
        BF_CASE(1) BF_CASE(2) BF_CASE(3) BF_CASE(4) BF_CASE(5) BF_CASE(6)
        BF_CASE(7) BF_CASE(8) BF_CASE(9) BF_CASE(10) BF_CASE(11) BF_CASE(12)
#undef BF_CASE
    default: return BF_ERR_UNSUPPORTED;
    }
    BF_CUDA(cudaGetLastError());
    return BF_OK;
}

bf_status run_fir_fused(const Call &c, int planes, float sigma_s)
{
    FIRCoef g;
    fir_coefs((double)sigma_s, c.p.w, &g);
    dim3 grid((c.ca.W + 31) / 32, (c.ca.H + 31) / 32, planes);
    if (c.p.box_passes) {  // 32-row tiles
        const int key = c.p.box_passes * 16 + c.p.box_r;
        switch (key) {
#define BF_BOX(P, R) \
    case P * 16 + R: fir_fused<P * R, P><<<grid, 256, 0, c.s>>>(c.ca, g); break;
            BF_BOX(1, 1) BF_BOX(1, 2) BF_BOX(1, 3) BF_BOX(1, 4) BF_BOX(1, 5) BF_BOX(1, 6)
            BF_BOX(1, 7) BF_BOX(1, 8) BF_BOX(1, 9) BF_BOX(1, 10) BF_BOX(1, 11) BF_BOX(1, 12)
            BF_BOX(2, 1) BF_BOX(2, 2) BF_BOX(2, 3) BF_BOX(2, 4) BF_BOX(2, 5) BF_BOX(2, 6)
            BF_BOX(3, 1) BF_BOX(3, 2) BF_BOX(3, 3) BF_BOX(3, 4)
#undef BF_BOX
        default: return BF_ERR_UNSUPPORTED;
        }
        BF_CUDA(cudaGetLastError());
        return BF_OK;
    }
    if (c.p.fir_tile == 16) return launch_fir_fused<16>(c, planes, g);
    if (c.p.fir_tile == 64) return launch_fir_fused<64>(c, planes, g);
    return launch_fir_fused<32>(c, planes, g);
}

template <int MODE>
bf_status run_cols(const Call &c, int planes, int W, float sigma_s)
{
    if (c.p.spatial == BF_SPATIAL_BOX) return BF_ERR_UNSUPPORTED;
    if (c.p.spatial == BF_SPATIAL_FIR) {
        FIRCoef g;
        fir_coefs((double)sigma_s, c.p.w, &g);
        bf_status st = BF_ERR_UNSUPPORTED;
        switch (c.p.w) {
#define BF_CASE(WW) \
    case WW: st = launch_col_fir_w<WW, MODE>(c.ca, g, planes, c.s); break;
            BF_CASE(1) BF_CASE(2) BF_CASE(3) BF_CASE(4) BF_CASE(5) BF_CASE(6)
            BF_CASE(7) BF_CASE(8) BF_CASE(9) BF_CASE(10) BF_CASE(11) BF_CASE(12)
#undef BF_CASE
        default: break;
        }
        if (st != BF_OK) return st;
    } else {
        const int strips = (W + 7) / 8;
        if (c.p.col_tc == 2) {
            IIRCoef cc;
            deriche_coefs((double)sigma_s, COL_C, &cc);
            UMat um;
            umma_mats((double)sigma_s, &um);
            if constexpr (MODE != MODE_JOINT)
                BF_CUDA(cudaFuncSetAttribute(col_tc5<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             TC5_SMEM_BYTES));
            cudaLaunchConfig_t cfg;
            std::memset(&cfg, 0, sizeof cfg);
            cfg.gridDim = dim3(strips * c.p.CL, planes, 1);
            cfg.blockDim = dim3(256, 1, 1);
            cfg.dynamicSmemBytes = TC5_SMEM_BYTES;
            cfg.stream = c.s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = (unsigned)c.p.CL;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if constexpr (MODE != MODE_JOINT) BF_CUDA(cudaLaunchKernelEx(&cfg, col_tc5<MODE>, c.ca, cc, um));
            BF_CUDA(cudaGetLastError());
            return BF_OK;
        }
        const bool tcore = c.p.col_tc != 0;
        IIRCoef cc;
        deriche_coefs((double)sigma_s, tcore ? TC_C : COL_C, &cc);
        TCMat tm;
        if (tcore) tc_mats((double)sigma_s, &tm);
        // the CUDA-core pass: the channel tiles, and for the saving forward its dp, dq ([2 C][256])
        const size_t smem = tcore ? sizeof(float) * COL_TILE_BUFS * COL_TILE_FLOATS
                                  : sizeof(float) * (COL_TILE_BUFS * COL_TILE_FLOATS +
                                                     (MODE == MODE_SAVE ? 2 * COL_C * 256 : 0) +
                                                     (MODE == MODE_FWD ? COL_U_FLOATS : 0));
        if constexpr (MODE != MODE_JOINT) {
            if (tcore)
                BF_CUDA(cudaFuncSetAttribute(col_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        }
        // the column pass for up to 4096 rows, or its instantiation for 16-CTA clusters
        auto col_kernel = c.p.CL > 8 ? col_iir<COL_C, MODE, COL_MAX_CTAS> : col_iir<COL_C, MODE, 8>;
        if (!tcore) BF_CUDA(cudaFuncSetAttribute(col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaLaunchConfig_t cfg;
        std::memset(&cfg, 0, sizeof cfg);
        cfg.gridDim = dim3(strips * c.p.CL, planes, 1);
        cfg.blockDim = dim3(256, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = c.s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)c.p.CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if constexpr (MODE != MODE_JOINT) {
            if (tcore) BF_CUDA(cudaLaunchKernelEx(&cfg, col_tc<MODE>, c.ca, cc, tm));
        }
        if (!tcore) {
            if (c.p.CL > 8) {
                // a column of more than 4096 rows: a cluster beyond the portable 8 CTAs, if the
                // device can hold one with this kernel's resources
                BF_CUDA(cudaFuncSetAttribute(col_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
                int nclusters = 0;
                if (cudaOccupancyMaxActiveClusters(&nclusters, col_kernel, &cfg) != cudaSuccess || nclusters < 1) {
                    cudaGetLastError();
                    return BF_ERR_UNSUPPORTED;
                }
            }
            BF_CUDA(cudaLaunchKernelEx(&cfg, col_kernel, c.ca, cc));
        }
    }
    BF_CUDA(cudaGetLastError());
    return BF_OK;
}

}  // namespace

extern "C" {

void bf_gp_default_opts(bf_gp_opts *opts)
{
    if (!opts) return;
    std::memset(opts, 0, sizeof *opts);
    opts->order = 20;
    opts->spatial = BF_SPATIAL_AUTO;
    opts->centre = BF_CENTRE_MEAN;
    opts->fir_halfwidth = 0;
    opts->t_c = 0.0;
}

const char *bf_status_string(bf_status s)
{
    switch (s) {
    case BF_OK: return "BF_OK";
    case BF_ERR_INVALID_ARG: return "BF_ERR_INVALID_ARG";
    case BF_ERR_WORKSPACE: return "BF_ERR_WORKSPACE";
    case BF_ERR_CUDA: return "BF_ERR_CUDA";
    case BF_ERR_UNSUPPORTED: return "BF_ERR_UNSUPPORTED";
    case BF_ERR_TIMEOUT: return "BF_ERR_TIMEOUT";
    }
    return "BF_ERR_UNKNOWN";
}

const char *bf_gp_last_cuda_error(void) { return g_cuda_err; }

int bf_gp_version(void) { return 100; }

bf_status bf_gp_workspace_size(int planes, int H, int W, float sigma_s, const bf_gp_opts *opts, size_t *bytes)
{
    if (!bytes) return BF_ERR_INVALID_ARG;
    bf_gp_opts d;
    if (!opts) {
        bf_gp_default_opts(&d);
        opts = &d;
    }
    Plan p;
    bf_status st = make_plan(planes, H, W, sigma_s, opts, &p);
    if (st != BF_OK) return st;
    *bytes = p.total;
    return BF_OK;
}

// The forward filter.  With src given, f is device memory the statistics
// pass fills from src (mapped host memory) before the other passes read it.
static bf_status forward_impl(const float *f, float *y, int planes, int H, int W, int pitch, float sigma_s,
                              float sigma_r, const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream,
                              const float *src, float *f_fill)
{
    Call c;
    bf_status st = prepare(f, y, planes, H, W, pitch, sigma_s, sigma_r, opts, ws, ws_bytes, stream, true, &c);
    if (st != BF_OK) return st;
    st = run_stats(c, planes, H, W, pitch, sigma_s, sigma_r, opts, 0, src, f_fill);
    if (st != BF_OK) return st;
    if (c.p.spatial == BF_SPATIAL_BOX) {
        if (opts->fir_two_pass) return BF_ERR_UNSUPPORTED;
        return run_fir_fused(c, planes, sigma_s);
    }
    if (c.p.spatial == BF_SPATIAL_FIR && opts->fir_two_pass == 0) return run_fir_fused(c, planes, sigma_s);
    st = run_rows<MODE_FWD>(c, planes, sigma_s);
    if (st == BF_OK) st = run_cols<MODE_FWD>(c, planes, W, sigma_s);
    return st;
}

bf_status bf_gp_forward(const float *f, float *y, int planes, int H, int W, int pitch, float sigma_s, float sigma_r,
                        const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream)
{
    return forward_impl(f, y, planes, H, W, pitch, sigma_s, sigma_r, opts, ws, ws_bytes, stream, nullptr, nullptr);
}

bf_status bf_gp_joint_workspace_size(int planes, int H, int W, float sigma_s, const bf_gp_opts *opts,
                                     size_t *bytes)
{
    if (!bytes) return BF_ERR_INVALID_ARG;
    bf_gp_opts d;
    if (!opts) {
        bf_gp_default_opts(&d);
        opts = &d;
    }
    Plan p;
    bf_status st = make_plan(planes, H, W, sigma_s, opts, &p, 1);
    if (st != BF_OK) return st;
    *bytes = p.total;
    return BF_OK;
}

bf_status bf_gp_forward_joint(const float *f, const float *g, float *y, int planes, int H, int W, int pitch,
                              float sigma_s, float sigma_r, const bf_gp_opts *opts, void *ws, size_t ws_bytes,
                              void *stream)
{
    if (!f || !g) return BF_ERR_INVALID_ARG;
    Call c;
    bf_status st = prepare(g, y, planes, H, W, pitch, sigma_s, sigma_r, opts, ws, ws_bytes, stream, true, &c, f);
    if (st != BF_OK) return st;
    // statistics of the guide; a constant guide is filtered (every range weight 1)
    st = run_stats(c, planes, H, W, pitch, sigma_s, sigma_r, opts, 3);
    if (st == BF_OK) st = run_rows<MODE_JOINT>(c, planes, sigma_s);
    if (st == BF_OK) st = run_cols<MODE_JOINT>(c, planes, W, sigma_s);
    return st;
}

bf_status bf_gp_phase_stats(const float *f, int planes, int H, int W, int pitch, float sigma_s, float sigma_r,
                            const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream)
{
    Call c;
    bf_status st = prepare(f, nullptr, planes, H, W, pitch, sigma_s, sigma_r, opts, ws, ws_bytes, stream, false, &c);
    if (st != BF_OK) return st;
    return run_stats(c, planes, H, W, pitch, sigma_s, sigma_r, opts, 0);
}

bf_status bf_gp_phase_rows(const float *f, int planes, int H, int W, int pitch, float sigma_s, float sigma_r,
                           const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream)
{
    Call c;
    bf_status st = prepare(f, nullptr, planes, H, W, pitch, sigma_s, sigma_r, opts, ws, ws_bytes, stream, false, &c);
    if (st != BF_OK) return st;
    return run_rows<MODE_FWD>(c, planes, sigma_s);
}

bf_status bf_gp_phase_cols(const float *f, float *y, int planes, int H, int W, int pitch, float sigma_s,
                           float sigma_r, const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream)
{
    Call c;
    bf_status st = prepare(f, y, planes, H, W, pitch, sigma_s, sigma_r, opts, ws, ws_bytes, stream, true, &c);
    if (st != BF_OK) return st;
    return run_cols<MODE_FWD>(c, planes, W, sigma_s);
}

bf_status bf_gp_forward_train(const float *f, float *y, float *saved, int planes, int H, int W, int pitch,
                              float sigma_s, float sigma_r, const bf_gp_opts *opts, void *ws, size_t ws_bytes,
                              void *stream)
{
    if (!saved) return BF_ERR_INVALID_ARG;
    Call c;
    bf_status st = prepare(f, y, planes, H, W, pitch, sigma_s, sigma_r, opts, ws, ws_bytes, stream, true, &c);
    if (st != BF_OK) return st;
    c.ca.saved = saved;
    st = run_stats(c, planes, H, W, pitch, sigma_s, sigma_r, opts, 1);
    if (st == BF_OK) st = run_rows<MODE_FWD>(c, planes, sigma_s);
    if (st == BF_OK) st = run_cols<MODE_SAVE>(c, planes, W, sigma_s);
    return st;
}

bf_status bf_gp_backward(const float *f, const float *grad_y, const float *saved, float *grad_f,
                         float *grad_sigma_r, int planes, int H, int W, int pitch, float sigma_s, float sigma_r,
                         const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream)
{
    if (!grad_y || !saved) return BF_ERR_INVALID_ARG;
    Call c;
    bf_status st = prepare(f, grad_f, planes, H, W, pitch, sigma_s, sigma_r, opts, ws, ws_bytes, stream, true, &c);
    if (st != BF_OK) return st;
    bf_gp_opts d;
    if (!opts) {
        bf_gp_default_opts(&d);
        opts = &d;
    }
    c.ra.gy = grad_y;
    c.ra.saved = saved;
    c.ca.gy = grad_y;
    c.ca.saved = const_cast<float *>(saved);
    st = run_stats(c, planes, H, W, pitch, sigma_s, sigma_r, opts, 1);
    if (st == BF_OK) st = run_rows<MODE_ADJ>(c, planes, sigma_s);
    if (st == BF_OK) st = run_cols<MODE_ADJ>(c, planes, W, sigma_s);
    if (st != BF_OK) return st;
    // bands of about 2048 pixels, at least one row each
    const int rows_per_band = std::max(1, 2048 / std::max(1, W));
    dim3 grid((unsigned)((H + rows_per_band - 1) / rows_per_band), planes);
    grad_finish<<<grid, 256, 0, c.s>>>(grad_f, c.acc, c.pp, H, W, pitch, opts->centre == BF_CENTRE_MEAN ? 1 : 0,
                                       (double)sigma_r, grad_sigma_r);
    BF_CUDA(cudaGetLastError());
    return BF_OK;
}

}  // extern "C"

// Scratch for bf_gp_forward_noalloc: a static device array, so the entry
// point needs neither a caller workspace nor an allocation.  Host code may
// not use the symbol itself as a device pointer; its device address is looked
// up once per device with cudaGetSymbolAddress (that device current) and cached,
// and looked up again when the cached one no longer names device memory of that
// device (a new context after cudaDeviceReset).
static __device__ __align__(256) unsigned char g_noalloc_scratch[BF_GP_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
}  // namespace

extern "C" {

bf_status bf_gp_forward_noalloc(const float *f, float *y, int planes, int H, int W, int pitch, float sigma_s,
                                float sigma_r, const bf_gp_opts *opts, void *stream)
{
    size_t need = 0;
    bf_status st = bf_gp_workspace_size(planes, H, W, sigma_s, opts, &need);
    if (st != BF_OK) return st;
    if (need > (size_t)BF_GP_NOALLOC_SCRATCH_BYTES) {
        snprintf(g_cuda_err, sizeof g_cuda_err,
                 "bf_gp_forward_noalloc: request needs %zu bytes of scratch; the static scratch holds %u", need,
                 (unsigned)BF_GP_NOALLOC_SCRATCH_BYTES);
        return BF_ERR_WORKSPACE;
    }
    int dev = -1;
    BF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return BF_ERR_UNSUPPORTED;
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        base = g_noalloc_ptr[dev];
        if (base) {
            // the cached address belongs to the context it was looked up in: after a
            // cudaDeviceReset the module is loaded again and the array may move
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, base) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
                at.device != dev || at.devicePointer != base) {
                (void)cudaGetLastError();
                base = nullptr;
            }
        }
        if (!base) {
            BF_CUDA(cudaGetSymbolAddress(&base, g_noalloc_scratch));
            g_noalloc_ptr[dev] = base;
        }
    }
    return bf_gp_forward(f, y, planes, H, W, pitch, sigma_s, sigma_r, opts, base,
                         (size_t)BF_GP_NOALLOC_SCRATCH_BYTES, stream);
}

bf_status bf_gp_host_workspace_size(int planes, int H, int W, float sigma_s, const bf_gp_opts *opts, size_t *bytes)
{
    size_t b = 0;
    bf_status st = bf_gp_workspace_size(planes, H, W, sigma_s, opts, &b);
    if (st != BF_OK) return st;
    *bytes = align_up(b, 256) + 2 * align_up(sizeof(float) * (size_t)planes * H * W, 256);
    return BF_OK;
}

// Device address of the host range [p, p + bytes) when both of its ends lie in
// pinned host memory mapped into the device's address space (cudaHostAlloc,
// or cudaHostRegister with the mapped flag) at consistent addresses; nullptr
// otherwise (pageable memory, device memory, a range that runs past a mapping).
static void *mapped_host_range(const void *p, size_t bytes)
{
    if (bytes == 0) return nullptr;
    cudaPointerAttributes a0, a1;
    const char *last = static_cast<const char *>(p) + bytes - 1;
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
        return nullptr;
    if (static_cast<char *>(a1.devicePointer) - static_cast<char *>(a0.devicePointer) != (ptrdiff_t)(bytes - 1))
        return nullptr;
    return a0.devicePointer;
}

bf_status bf_gp_forward_host(const float *f_host, float *y_host, int planes, int H, int W, float sigma_s,
                             float sigma_r, const bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream)
{
    if (!f_host || !y_host || !ws) return BF_ERR_INVALID_ARG;
    size_t need = 0, base = 0;
    bf_status st = bf_gp_host_workspace_size(planes, H, W, sigma_s, opts, &need);
    if (st != BF_OK) return st;
    st = bf_gp_workspace_size(planes, H, W, sigma_s, opts, &base);
    if (st != BF_OK) return st;
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < need) return BF_ERR_WORKSPACE;
    const size_t img = sizeof(float) * (size_t)planes * H * W;
    char *wsb = static_cast<char *>(ws);
    float *fd = reinterpret_cast<float *>(wsb + align_up(base, 256));
    float *yd = reinterpret_cast<float *>(wsb + align_up(base, 256) + align_up(img, 256));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // A mapped pinned result buffer is written by the last pass itself: its
    // stores travel to host memory while other CTAs are still computing,
    // instead of a device->host copy after the pass.
    float *ymap = (reinterpret_cast<uintptr_t>(y_host) & 3) == 0
                      ? static_cast<float *>(mapped_host_range(y_host, img))
                      : nullptr;
    // Likewise a mapped pinned input is read by the statistics pass itself,
    // which stores the device copy the other passes use.
    const float *fmap = (reinterpret_cast<uintptr_t>(f_host) & 3) == 0
                            ? static_cast<const float *>(mapped_host_range(f_host, img))
                            : nullptr;
    if (!fmap) BF_CUDA(cudaMemcpyAsync(fd, f_host, img, cudaMemcpyHostToDevice, s));
    st = forward_impl(fd, ymap ? ymap : yd, planes, H, W, W, sigma_s, sigma_r, opts, ws, base, stream, fmap,
                      fmap ? fd : nullptr);
    if (st != BF_OK) return st;
    if (!ymap) BF_CUDA(cudaMemcpyAsync(y_host, yd, img, cudaMemcpyDeviceToHost, s));
    BF_CUDA(cudaStreamSynchronize(s));
    return BF_OK;
}

bf_status bf_gp_get_device_status(const void *ws, void *stream, uint32_t *bits)
{
    if (!ws || !bits) return BF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BF_CUDA(cudaStreamSynchronize(s));
    BF_CUDA(cudaMemcpy(bits, ws, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return BF_OK;
}

bf_status bf_gp_get_device_counters(const void *ws, void *stream, unsigned long long *counters)
{
    if (!ws || !counters) return BF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BF_CUDA(cudaStreamSynchronize(s));
    BF_CUDA(cudaMemcpy(counters, static_cast<const char *>(ws) + 8, sizeof(unsigned long long) * NCOUNTERS,
                       cudaMemcpyDeviceToHost));
    return BF_OK;
}

bf_status bf_gp_get_plane_stats(const void *ws, int plane, void *stream, double *t_c, double *R)
{
    if (!ws || plane < 0) return BF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BF_CUDA(cudaStreamSynchronize(s));
    PlaneParams q;
    const char *src = static_cast<const char *>(ws) + HDR_BYTES + sizeof(PlaneParams) * (size_t)plane;
    BF_CUDA(cudaMemcpy(&q, src, sizeof q, cudaMemcpyDeviceToHost));
    if (t_c) *t_c = q.tc_d;
    if (R) *R = q.R_d;
    return BF_OK;
}

int bf_gp_order_for_tol(double sigma_r, double R, double eps)
{
    if (!(sigma_r > 0.0) || !(R >= 0.0) || !(eps > 0.0)) return -1;
    const int G = 257;
    for (int N = 0; N <= KMAX - 2; N += 2) {
        double worst = 0.0;
        for (int a = 0; a < G && worst <= eps; ++a) {
            const double tau = -R + 2.0 * R * a / (G - 1);
            for (int b = 0; b < G; ++b) {
                const double t = -R + 2.0 * R * b / (G - 1);
                const double x = tau * t / (sigma_r * sigma_r);
                double term = 1.0, sum = 0.0;
                for (int n = 0; n <= N; ++n) {
                    sum += term;
                    term *= x / (double)(n + 1);
                }
                const double gp = std::exp(-(tau * tau + t * t) / (2.0 * sigma_r * sigma_r)) * sum;
                const double g = std::exp(-(t - tau) * (t - tau) / (2.0 * sigma_r * sigma_r));
                worst = std::fmax(worst, std::fabs(g - gp));
            }
        }
        if (worst <= eps) return N;
    }
    return -1;
}

int bf_gp_order_fp32_limit(double sigma_s, double sigma_r, double R)
{
    if (!(sigma_s > 0.0) || !(sigma_r > 0.0) || !(R >= 0.0)) return -1;
    // the statistics pass's range test (flag BF_DEV_RANGE), one bit tighter
    const double s2 = std::isinf(sigma_r) ? 0.0 : (R / sigma_r) * (R / sigma_r);
    const float s2f = (float)s2;
    if (0.3606738f * s2f > 119.f) return -1;
    const float e0 = std::fmax(0.f, std::ceil(0.7213475f * s2f - 120.f));
    const float gain = 2.f * std::log2(2.6f * (float)sigma_s + 2.f);
    int best = -1;
    float top = 0.f;  // max over the channels so far of log2(beta_k max_u E u^k); channel 0 gives 0
    double beta = 1.0;
    for (int k = 1; k <= KMAX - 1; ++k) {
        if (k >= 2) beta *= s2 * (1.0 / (double)k);
        if (beta > 0.0) {
            const float u2 = std::fmin(1.f, (float)k / s2f);
            top = std::fmax(top, std::log2((float)beta) - 0.7213475f * s2f * u2 + 0.5f * (float)k * std::log2(u2));
        }
        const int N = k - 1, K = k + 1;  // channels 0..k
        if (N % 2 == 0 && e0 + top + gain + 2.f * std::log2((float)K) <= 123.f) best = N;
    }
    return best;
}

}  // extern "C"

// ---------------------------------------------------------------- batched

constexpr int BATCH_STREAMS = BF_GP_BATCH_STREAMS;  // planes of a batch filtered concurrently

struct bf_gp_plan {
    std::vector<BatchPlane> bp;  // device pointers to ws filled at upload
    std::vector<IIRCoef> coef;
    std::vector<int> pre_stats, pre_rows, pre_cols;  // pre_cols over col_order
    std::vector<int> col_order;                      // planes sorted by column cluster size
    std::vector<int> grp_cl, grp_start, grp_count;   // column launches: cluster size, first item, items
    std::vector<size_t> plane_off;  // byte offset of each plane's channel planes
    int n = 0, CLmax = 1, total_stats = 0, total_rows = 0, total_strips = 0;
    int centre_given = 0;
    double tc_given = 0.0;
    size_t off_params = 0, off_part = 0, off_tables = 0, off_planes = 0, total = 0;
    size_t tables_bytes = 0;
    const void *uploaded_ws = nullptr;
    // filtering: every plane through the single-image launches (its own sub-workspace at
    // off_planes + sub_off[i]), spread over the plan's streams
    std::vector<bf_gp_plane> specs;
    bf_gp_opts base;
    std::vector<int> engine;       // per plane: base.engine, or the autotuner's choice (bf_gp_batched_plan_tune)
    std::vector<int> row_threads;  // per plane: base.row_threads, or the autotuner's choice
    std::vector<size_t> sub_off, sub_bytes;
    size_t off_statusofs = 0;  // in the tables: byte offset of every plane's status word, n x uint64
    // persistent launch (bf_gp_batched_persistent): per-plane descriptors and coefficients, the work
    // items in dependency order, the work and readiness counters; tables at off_ptables in ws
    std::vector<PersistPlane> ppl;
    std::vector<IIRCoef> pcrow, pccol;
    std::vector<TCMat> ptm;
    std::vector<int4> pitems;  // in the order of the launch (set at upload, when the grid is known)
    std::vector<int4> pstats, pfinal, prows, pcols;  // per kind, plane by plane
    int pcl = 1;               // cluster size of the persistent launch
    bool persist_ok = false;   // every plane within its kernels' limits (rows of at most 4096 samples)
    size_t off_ptables = 0, ptables_bytes = 0, off_pitems = 0, off_pcount = 0;
    long long wait_cycles = 1ll << 32;  // about two seconds at 2 GHz
    int starve_plane = -1;
    int pclusters = 0;         // clusters resident at once (found at upload; 0: none fits)
    int nstreams = 0;
    cudaStream_t streams[BATCH_STREAMS] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[BATCH_STREAMS] = {};
    ~bf_gp_plan()
    {
        for (int i = 0; i < nstreams; ++i) {
            if (ev_join[i]) cudaEventDestroy(ev_join[i]);
            if (streams[i]) cudaStreamDestroy(streams[i]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
    }
};

extern "C" {

}  // extern "C"

namespace {

// The persistent launch's tables: each plane's descriptor (offsets into its single-image
// workspace), its coefficients, and its work items: statistics partials (stat_m per CTA,
// pcl CTAs per item), its finalisation, its row groups (row_m per CTA), its column strips
// (pcl / G per item, G CTAs per strip).  The launch order of the items is set at upload
// (order_items).  Planes whose rows exceed 4096 samples are outside the row pass's 256-thread
// CTAs, and columns longer than 4096 rows outside an 8-CTA cluster: the plan then has no
// persistent form.
bf_status build_persistent(bf_gp_plan *pl, const bf_gp_plane *planes, const bf_gp_opts *opts)
{
    const int n = pl->n;
    pl->persist_ok = true;
    int clmax = 1;
    for (int i = 0; i < n; ++i) {
        if (planes[i].W > 4096) pl->persist_ok = false;
        clmax = std::max(clmax, (planes[i].H + COL_ROWS_PER_CTA - 1) / COL_ROWS_PER_CTA);
    }
    if (clmax > 8) pl->persist_ok = false;
    if (!pl->persist_ok) return BF_OK;
    pl->pcl = next_pow2(clmax);
    pl->ppl.resize(n);
    pl->pcrow.resize(n);
    pl->pccol.resize(n);
    pl->ptm.resize(n);
    std::vector<int4> stats, fin, rows, cols;
    for (int i = 0; i < n; ++i) {
        const bf_gp_plane &q = planes[i];
        bf_gp_opts o = *opts;
        o.order = q.order;
        o.spatial = BF_SPATIAL_IIR;
        o.engine = 0;
        o.row_threads = 0;
        Plan pp;
        bf_status st = make_plan(1, q.H, q.W, q.sigma_s, &o, &pp);
        if (st != BF_OK) return st;
        PersistPlane &d = pl->ppl[i];
        std::memset(&d, 0, sizeof d);
        d.f = q.f;
        d.y = q.y;
        d.off_params = (long long)pp.off_params;
        d.off_part = (long long)pp.off_part;
        d.off_planes = (long long)pp.off_planes;
        d.H = q.H;
        d.W = q.W;
        d.pitch = q.pitch;
        d.Wp = pp.Wp;
        d.K = pp.K;
        d.N = pp.N;
        d.wpr = pp.wpr;
        d.nblk = pp.nblk;
        d.rows_per_block = pp.rows_per_block;
        const int rows_per_cta = 8 / pp.wpr;  // 256 threads: 8 warps, wpr per row
        d.rowgroups = (q.H + rows_per_cta - 1) / rows_per_cta;
        d.strips = (q.W + 7) / 8;
        d.G = next_pow2(pp.CL);
        // per item, a CTA takes about 32K pixels of statistics and 16K pixels of rows
        const long long blk_px = (long long)pp.rows_per_block * q.W, grp_px = (long long)rows_per_cta * q.W;
        d.stat_m = (int)std::min<long long>(64, std::max<long long>(1, (32768 + blk_px - 1) / blk_px));
        d.row_m = (int)std::min<long long>(16, std::max<long long>(1, (16384 + grp_px - 1) / grp_px));
        d.sigma_s = q.sigma_s;
        d.sigma_r = q.sigma_r;
        deriche_coefs((double)q.sigma_s, TC_C, &pl->pcrow[i]);
        deriche_coefs((double)q.sigma_s, COL_C, &pl->pccol[i]);
        tc_mats((double)q.sigma_s, &pl->ptm[i]);
        const int c = pl->pcl;
        const int su = c * d.stat_m, ru = c * d.row_m;  // units per item
        for (int u = 0; u < d.nblk; u += su) stats.push_back(make_int4(PITEM_STATS, i, u, std::min(su, d.nblk - u)));
        fin.push_back(make_int4(PITEM_FINAL, i, 0, 1));
        for (int u = 0; u < d.rowgroups; u += ru)
            rows.push_back(make_int4(PITEM_ROWS, i, u, std::min(ru, d.rowgroups - u)));
        const int per = c / d.G;  // strips per column item
        for (int u = 0; u < d.strips; u += per) cols.push_back(make_int4(PITEM_COLS, i, u, std::min(per, d.strips - u)));
    }
    pl->pstats = stats;
    pl->pfinal = fin;
    pl->prows = rows;
    pl->pcols = cols;
    pl->pitems.resize(stats.size() + fin.size() + rows.size() + cols.size());
    size_t o = 0;
    o += sizeof(PersistPlane) * n;
    o = align_up(o, 16) + sizeof(IIRCoef) * n;
    o = align_up(o, 16) + sizeof(IIRCoef) * n;
    o = align_up(o, 16) + sizeof(TCMat) * n;
    pl->off_pitems = align_up(o, 16);
    o = pl->off_pitems + sizeof(int4) * pl->pitems.size();
    pl->off_pcount = align_up(o, 16);
    pl->ptables_bytes = pl->off_pcount + sizeof(int) * (1 + 3 * (size_t)n);
    pl->off_ptables = align_up(pl->total, 256);
    pl->total = pl->off_ptables + pl->ptables_bytes;
    return BF_OK;
}

// The persistent launch's shape: one cluster of pcl CTAs of 256 threads (the grid is set by the caller).
void persist_config(const bf_gp_plan *pl, cudaStream_t s, cudaLaunchConfig_t *cfg, cudaLaunchAttribute *attr)
{
    std::memset(cfg, 0, sizeof *cfg);
    cfg->blockDim = dim3(256, 1, 1);
    cfg->gridDim = dim3((unsigned)pl->pcl, 1, 1);
    cfg->dynamicSmemBytes = sizeof(float) * (COL_TILE_BUFS * COL_TILE_FLOATS + COL_U_FLOATS);
    cfg->stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)pl->pcl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg->attrs = attr;
    cfg->numAttrs = 1;
}

// Copies the persistent tables (with this workspace's plane addresses) into ws, waits, and
// finds how many clusters are resident at once.
// The launch's item order: all statistics partials, all centres and scales, then the row items
// plane after plane, each plane's column items following once `lag` row items have come after its
// last one (or at the end).  Every item comes after the items it waits for.
void order_items(bf_gp_plan *pl, int lag)
{
    std::vector<int4> &o = pl->pitems;
    o.clear();
    o.insert(o.end(), pl->pstats.begin(), pl->pstats.end());
    o.insert(o.end(), pl->pfinal.begin(), pl->pfinal.end());
    size_t r = 0, c = 0;
    std::vector<std::pair<int, long long>> pending;  // (plane, row items placed when its rows ended)
    long long placed = 0;
    auto flush = [&](bool all) {
        while (!pending.empty() && (all || placed - pending.front().second >= lag)) {
            const int p = pending.front().first;
            while (c < pl->pcols.size() && pl->pcols[c].y == p) o.push_back(pl->pcols[c++]);
            pending.erase(pending.begin());
        }
    };
    while (r < pl->prows.size()) {
        const int p = pl->prows[r].y;
        while (r < pl->prows.size() && pl->prows[r].y == p) {
            o.push_back(pl->prows[r++]);
            ++placed;
            flush(false);
        }
        pending.emplace_back(p, placed);
    }
    flush(true);
}

bf_status upload_persistent(bf_gp_plan *pl, char *wsb, cudaStream_t s)
{
    if (!pl->persist_ok) return BF_OK;
    const int n = pl->n;
    std::vector<char> img(pl->off_pcount, 0);
    std::vector<PersistPlane> d = pl->ppl;
    for (int i = 0; i < n; ++i) d[i].ws = wsb + pl->off_planes + pl->sub_off[i];
    size_t o = 0;
    std::memcpy(img.data() + o, d.data(), sizeof(PersistPlane) * n);
    o += sizeof(PersistPlane) * n;
    o = align_up(o, 16);
    std::memcpy(img.data() + o, pl->pcrow.data(), sizeof(IIRCoef) * n);
    o += sizeof(IIRCoef) * n;
    o = align_up(o, 16);
    std::memcpy(img.data() + o, pl->pccol.data(), sizeof(IIRCoef) * n);
    o += sizeof(IIRCoef) * n;
    o = align_up(o, 16);
    std::memcpy(img.data() + o, pl->ptm.data(), sizeof(TCMat) * n);
    o += sizeof(TCMat) * n;
    BF_CUDA(cudaMemcpyAsync(wsb + pl->off_ptables, img.data(), img.size(), cudaMemcpyHostToDevice, s));
    BF_CUDA(cudaStreamSynchronize(s));
    // how many clusters of the launch's shape are resident at once on this device
    const size_t smem = sizeof(float) * (COL_TILE_BUFS * COL_TILE_FLOATS + COL_U_FLOATS);
    BF_CUDA(cudaFuncSetAttribute(batched_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    persist_config(pl, s, &cfg, attr);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, batched_persistent, &cfg) != cudaSuccess) {
        cudaGetLastError();
        nclusters = 0;
    }
    pl->pclusters = nclusters;
    // column items two rounds of the grid after their plane's last row item
    order_items(pl, 2ll * std::max(1, nclusters));
    BF_CUDA(cudaMemcpyAsync(wsb + pl->off_ptables + pl->off_pitems, pl->pitems.data(),
                            sizeof(int4) * pl->pitems.size(), cudaMemcpyHostToDevice, s));
    BF_CUDA(cudaStreamSynchronize(s));
    return BF_OK;
}

PersistArgs persist_args(const bf_gp_plan *pl, char *wsb)
{
    const int n = pl->n;
    char *tb = wsb + pl->off_ptables;
    PersistArgs a;
    std::memset(&a, 0, sizeof a);
    size_t o = 0;
    a.pl = reinterpret_cast<const PersistPlane *>(tb + o);
    o = align_up(o + sizeof(PersistPlane) * n, 16);
    a.crow = reinterpret_cast<const IIRCoef *>(tb + o);
    o = align_up(o + sizeof(IIRCoef) * n, 16);
    a.ccol = reinterpret_cast<const IIRCoef *>(tb + o);
    o = align_up(o + sizeof(IIRCoef) * n, 16);
    a.tm = reinterpret_cast<const TCMat *>(tb + o);
    a.items = reinterpret_cast<const int4 *>(tb + pl->off_pitems);
    a.work = reinterpret_cast<int *>(tb + pl->off_pcount);
    a.ready = a.work + 1;
    a.nitems = (int)pl->pitems.size();
    a.centre_given = pl->centre_given;
    a.tc_given = pl->tc_given;
    a.wait_cycles = pl->wait_cycles;
    a.starve_plane = pl->starve_plane;
    return a;
}

}  // namespace

extern "C" {

bf_status bf_gp_batched_plan_create(const bf_gp_plane *planes, int n, const bf_gp_opts *opts, bf_gp_plan **out)
{
    if (!planes || n < 1 || !out) return BF_ERR_INVALID_ARG;
    bf_gp_opts d;
    if (!opts) {
        bf_gp_default_opts(&d);
        opts = &d;
    }
    bf_status st = check_opts(opts);
    if (st != BF_OK) return st;
    if (opts->spatial == BF_SPATIAL_FIR || opts->spatial == BF_SPATIAL_BOX)
        return BF_ERR_UNSUPPORTED;  // batched planes use the recursive filter
    bf_gp_plan *pl = new (std::nothrow) bf_gp_plan;
    if (!pl) return BF_ERR_INVALID_ARG;
    pl->n = n;
    pl->centre_given = opts->centre == BF_CENTRE_GIVEN ? 1 : 0;
    pl->tc_given = opts->t_c;
    pl->bp.resize(n);
    pl->coef.resize(n);
    pl->pre_stats.assign(n + 1, 0);
    pl->pre_rows.assign(n + 1, 0);
    pl->pre_cols.assign(n + 1, 0);
    pl->plane_off.resize(n);
    size_t planes_bytes = 0;
    for (int i = 0; i < n; ++i) {
        const bf_gp_plane &q = planes[i];
        bf_gp_opts o = *opts;
        o.order = q.order;
        o.spatial = BF_SPATIAL_IIR;
        Plan pp;
        st = (q.f && q.y && q.pitch >= q.W && q.sigma_r > 0.f) ? make_plan(1, q.H, q.W, q.sigma_s, &o, &pp)
                                                                  : BF_ERR_INVALID_ARG;
        if (st != BF_OK) {
            delete pl;
            return st;
        }
        BatchPlane &b = pl->bp[i];
        std::memset(&b, 0, sizeof b);
        b.f = q.f;
        b.y = q.y;
        b.H = q.H;
        b.W = q.W;
        b.pitch = q.pitch;
        b.Wp = pp.Wp;
        b.K = pp.K;
        b.N = pp.N;
        b.T = pp.T;
        b.nblk = pp.nblk;
        b.rows_per_block = pp.rows_per_block;
        b.sigma_s = q.sigma_s;
        b.sigma_r = q.sigma_r;
        deriche_coefs((double)q.sigma_s, ROW_C, &pl->coef[i]);
        const int rows_per_cta = 256 / pp.T;
        pl->pre_stats[i + 1] = pl->pre_stats[i] + pp.nblk;
        pl->pre_rows[i + 1] = pl->pre_rows[i] + (q.H + rows_per_cta - 1) / rows_per_cta;
        pl->CLmax = std::max(pl->CLmax, pp.CL);
        pl->plane_off[i] = planes_bytes;
        planes_bytes = align_up(planes_bytes + pp.total, 256);  // the plane's single-image workspace
    }
    pl->specs.assign(planes, planes + n);
    pl->base = *opts;
    pl->engine.assign(n, opts->engine);
    pl->row_threads.assign(n, opts->row_threads);
    pl->sub_off = pl->plane_off;
    pl->sub_bytes.resize(n);
    for (int i = 0; i < n; ++i)
        pl->sub_bytes[i] = (i + 1 < n ? pl->plane_off[i + 1] : planes_bytes) - pl->plane_off[i];
    // column work: planes sorted by cluster size, one launch per size
    pl->col_order.resize(n);
    for (int i = 0; i < n; ++i) pl->col_order[i] = i;
    auto cl_of = [&](int i) { return (planes[i].H + COL_ROWS_PER_CTA - 1) / COL_ROWS_PER_CTA; };
    std::stable_sort(pl->col_order.begin(), pl->col_order.end(), [&](int x, int y) { return cl_of(x) < cl_of(y); });
    for (int j = 0; j < n; ++j) {
        const int i = pl->col_order[j];
        pl->pre_cols[j + 1] = pl->pre_cols[j] + (planes[i].W + 7) / 8;
        if (pl->grp_cl.empty() || pl->grp_cl.back() != cl_of(i)) {
            pl->grp_cl.push_back(cl_of(i));
            pl->grp_start.push_back(pl->pre_cols[j]);
            pl->grp_count.push_back(0);
        }
        pl->grp_count.back() += (planes[i].W + 7) / 8;
    }
    pl->total_stats = pl->pre_stats[n];
    pl->total_rows = pl->pre_rows[n];
    pl->total_strips = pl->pre_cols[n];
    size_t off = HDR_BYTES;
    pl->off_params = off;
    off = align_up(off + sizeof(PlaneParams) * (size_t)n, 256);
    pl->off_part = off;
    off = align_up(off + sizeof(StatPartial) * (size_t)pl->total_stats, 256);
    pl->off_tables = off;
    pl->tables_bytes = sizeof(BatchPlane) * n + sizeof(IIRCoef) * n + sizeof(int) * (3 * (n + 1) + n);
    pl->tables_bytes = align_up(pl->tables_bytes, 8);
    pl->off_statusofs = pl->tables_bytes;
    pl->tables_bytes += sizeof(unsigned long long) * (size_t)n;
    off = align_up(off + pl->tables_bytes, 256);
    pl->off_planes = off;
    pl->total = off + planes_bytes;
    st = build_persistent(pl, planes, opts);
    if (st != BF_OK) {
        delete pl;
        return st;
    }
    pl->nstreams = std::min(n, BATCH_STREAMS);
    bool ok = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < pl->nstreams; ++i)
        ok = cudaStreamCreateWithFlags(&pl->streams[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&pl->ev_join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        delete pl;
        return BF_ERR_CUDA;
    }
    *out = pl;
    return BF_OK;
}

bf_status bf_gp_batched_plan_workspace(const bf_gp_plan *plan, size_t *bytes)
{
    if (!plan || !bytes) return BF_ERR_INVALID_ARG;
    *bytes = plan->total;
    return BF_OK;
}

namespace {

// Copies the plan's tables (descriptors with this workspace's plane pointers,
// filter coefficients, prefix sums) into ws and waits for the copy.
bf_status upload_tables(const bf_gp_plan *plan, char *wsb, cudaStream_t s)
{
    const int n = plan->n;
    std::vector<char> img(plan->tables_bytes);
    std::vector<BatchPlane> bp = plan->bp;
    for (int i = 0; i < n; ++i) bp[i].ws = reinterpret_cast<float *>(wsb + plan->off_planes + plan->plane_off[i]);
    size_t o = 0;
    std::memcpy(img.data() + o, bp.data(), sizeof(BatchPlane) * n);
    o += sizeof(BatchPlane) * n;
    std::memcpy(img.data() + o, plan->coef.data(), sizeof(IIRCoef) * n);
    o += sizeof(IIRCoef) * n;
    std::memcpy(img.data() + o, plan->pre_stats.data(), sizeof(int) * (n + 1));
    o += sizeof(int) * (n + 1);
    std::memcpy(img.data() + o, plan->pre_rows.data(), sizeof(int) * (n + 1));
    o += sizeof(int) * (n + 1);
    std::memcpy(img.data() + o, plan->pre_cols.data(), sizeof(int) * (n + 1));
    o += sizeof(int) * (n + 1);
    std::memcpy(img.data() + o, plan->col_order.data(), sizeof(int) * n);
    for (int i = 0; i < n; ++i) {
        const unsigned long long so = (unsigned long long)(plan->off_planes + plan->sub_off[i]);  // status at 0
        std::memcpy(img.data() + plan->off_statusofs + sizeof(so) * (size_t)i, &so, sizeof so);
    }
    BF_CUDA(cudaMemcpyAsync(wsb + plan->off_tables, img.data(), plan->tables_bytes, cudaMemcpyHostToDevice, s));
    BF_CUDA(cudaStreamSynchronize(s));
    return BF_OK;
}

BatchArgs batch_args(const bf_gp_plan *plan, char *wsb)
{
    const int n = plan->n;
    const char *tb = wsb + plan->off_tables;
    BatchArgs b;
    b.bp = reinterpret_cast<const BatchPlane *>(tb);
    b.coef = reinterpret_cast<const IIRCoef *>(tb + sizeof(BatchPlane) * n);
    const int *pre = reinterpret_cast<const int *>(tb + sizeof(BatchPlane) * n + sizeof(IIRCoef) * n);
    b.pre_stats = pre;
    b.pre_rows = pre + (n + 1);
    b.pre_cols = pre + 2 * (n + 1);
    b.col_order = pre + 3 * (n + 1);
    b.cid0 = 0;
    b.pad = 0;
    b.pp = reinterpret_cast<PlaneParams *>(wsb + plan->off_params);
    b.part = reinterpret_cast<StatPartial *>(wsb + plan->off_part);
    b.status = reinterpret_cast<uint32_t *>(wsb);
    b.n = n;
    b.centre_given = plan->centre_given;
    b.tc_given = plan->tc_given;
    return b;
}

}  // namespace

bf_status bf_gp_batched_plan_upload(bf_gp_plan *plan, void *ws, size_t ws_bytes, void *stream)
{
    if (!plan || !ws) return BF_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < plan->total) return BF_ERR_WORKSPACE;
    bf_status st = upload_tables(plan, static_cast<char *>(ws), reinterpret_cast<cudaStream_t>(stream));
    if (st == BF_OK) st = upload_persistent(plan, static_cast<char *>(ws), reinterpret_cast<cudaStream_t>(stream));
    if (st != BF_OK) return st;
    plan->uploaded_ws = ws;
    return BF_OK;
}

bf_status bf_gp_batched_plan_stats_workspace(const bf_gp_plan *plan, size_t *bytes)
{
    if (!plan || !bytes) return BF_ERR_INVALID_ARG;
    *bytes = plan->off_planes;
    return BF_OK;
}

bf_status bf_gp_batched_plane_stats(const bf_gp_plan *plan, void *ws, size_t ws_bytes, void *stream, double *t_c,
                                    double *R)
{
    if (!plan || !ws) return BF_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < plan->off_planes) return BF_ERR_WORKSPACE;
    char *wsb = static_cast<char *>(ws);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    bf_status st = upload_tables(plan, wsb, s);
    if (st != BF_OK) return st;
    BF_CUDA(cudaMemsetAsync(wsb, 0, 8 + sizeof(unsigned long long) * NCOUNTERS, s));  // status word and counters
    BatchArgs b = batch_args(plan, wsb);
    batched_stats_partial<<<plan->total_stats, 256, 0, s>>>(b);
    batched_stats_finalize<<<plan->n, 256, 0, s>>>(b);
    BF_CUDA(cudaGetLastError());
    std::vector<PlaneParams> q(plan->n);
    BF_CUDA(cudaMemcpyAsync(q.data(), wsb + plan->off_params, sizeof(PlaneParams) * (size_t)plan->n,
                            cudaMemcpyDeviceToHost, s));
    BF_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < plan->n; ++i) {
        if (t_c) t_c[i] = q[i].tc_d;
        if (R) R[i] = q[i].R_d;
    }
    return BF_OK;
}

bf_status bf_gp_batched(const bf_gp_plan *plan, void *ws, size_t ws_bytes, void *stream)
{
    if (!plan || !ws) return BF_ERR_INVALID_ARG;
    if (ws != plan->uploaded_ws || ws_bytes < plan->total) return BF_ERR_WORKSPACE;
    const int n = plan->n;
    char *wsb = static_cast<char *>(ws);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // fork: the plan's streams start after the work already on `stream` (also under capture)
    BF_CUDA(cudaEventRecord(plan->ev_fork, s));
    for (int j = 0; j < plan->nstreams; ++j) BF_CUDA(cudaStreamWaitEvent(plan->streams[j], plan->ev_fork, 0));
    bf_status st = BF_OK;
    for (int i = 0; i < n && st == BF_OK; ++i) {
        const bf_gp_plane &q = plan->specs[i];
        bf_gp_opts o = plan->base;
        o.order = q.order;
        o.spatial = BF_SPATIAL_IIR;
        o.engine = plan->engine[i];
        o.row_threads = plan->row_threads[i];
        cudaStream_t si = plan->streams[i % plan->nstreams];
        Call c;
        st = prepare(q.f, q.y, 1, q.H, q.W, q.pitch, q.sigma_s, q.sigma_r, &o, wsb + plan->off_planes + plan->sub_off[i],
                     plan->sub_bytes[i], si, true, &c);
        if (st == BF_OK) st = run_stats(c, 1, q.H, q.W, q.pitch, q.sigma_s, q.sigma_r, &o, 0);
        if (st == BF_OK) st = run_rows<MODE_FWD>(c, 1, q.sigma_s);
        if (st == BF_OK) st = run_cols<MODE_FWD>(c, 1, q.W, q.sigma_s);
    }
    // join, then gather the planes' status words into the batch's
    for (int j = 0; j < plan->nstreams; ++j) {
        BF_CUDA(cudaEventRecord(plan->ev_join[j], plan->streams[j]));
        BF_CUDA(cudaStreamWaitEvent(s, plan->ev_join[j], 0));
    }
    if (st != BF_OK) return st;
    const unsigned long long *ofs =
        reinterpret_cast<const unsigned long long *>(wsb + plan->off_tables + plan->off_statusofs);
    gather_status<<<1, 256, 0, s>>>(reinterpret_cast<uint32_t *>(wsb), wsb, ofs, n);
    BF_CUDA(cudaGetLastError());
    return BF_OK;
}

bf_status bf_gp_batched_persistent(const bf_gp_plan *plan, void *ws, size_t ws_bytes, void *stream)
{
    if (!plan || !ws) return BF_ERR_INVALID_ARG;
    if (ws != plan->uploaded_ws || ws_bytes < plan->total) return BF_ERR_WORKSPACE;
    if (!plan->persist_ok) return BF_ERR_UNSUPPORTED;
    char *wsb = static_cast<char *>(ws);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    PersistArgs a = persist_args(plan, wsb);
    if (plan->pclusters < 1) return BF_ERR_UNSUPPORTED;
    const unsigned long long *ofs =
        reinterpret_cast<const unsigned long long *>(wsb + plan->off_tables + plan->off_statusofs);
    // the work counter, every plane's readiness counters, status word and counters start at zero
    BF_CUDA(cudaMemsetAsync(a.work, 0, sizeof(int) * (1 + 3 * (size_t)plan->n), s));
    zero_plane_status<<<(plan->n + 255) / 256, 256, 0, s>>>(wsb, ofs, plan->n);
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    persist_config(plan, s, &cfg, attr);
    cfg.gridDim = dim3((unsigned)(plan->pclusters * plan->pcl), 1, 1);  // the clusters resident at once
    BF_CUDA(cudaLaunchKernelEx(&cfg, batched_persistent, a));
    gather_status<<<1, 256, 0, s>>>(reinterpret_cast<uint32_t *>(wsb), wsb, ofs, plan->n);
    BF_CUDA(cudaGetLastError());
    return BF_OK;
}

bf_status bf_gp_batched_plan_set_wait(bf_gp_plan *plan, long long wait_cycles, int starve_plane)
{
    if (!plan || wait_cycles < 1 || starve_plane < -1 || starve_plane >= plan->n) return BF_ERR_INVALID_ARG;
    plan->wait_cycles = wait_cycles;
    plan->starve_plane = starve_plane;
    return BF_OK;
}

void bf_gp_batched_plan_destroy(bf_gp_plan *plan) { delete plan; }

// ------------------------------------------------------------------ autotuner
//
// The engines of the recursive filter (and the fused or two-pass form of the
// FIR filter) compute the same filter with different kernels; which is
// fastest depends on the shape (measured on GB300: the tensor-core row pass
// wins from 2048^2 up, the CUDA-core row pass on small and thin images).
// The tuner times every candidate on the caller's own buffers and keeps the
// winner per shape class for the life of the process.

}  // extern "C"

namespace {

// shape class: device, planes, H, W, pitch, resolved spatial operator, K, FIR half-width
using TuneKey = std::tuple<int, int, int, int, int, int, int, int>;
std::mutex g_tune_mutex;
std::map<TuneKey, bf_gp_opts> g_tune;

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" {

bf_status bf_gp_autotune(const float *f, float *y, int planes, int H, int W, int pitch, float sigma_s,
                         float sigma_r, bf_gp_opts *opts, void *ws, size_t ws_bytes, void *stream, int reps,
                         float *ms)
{
    if (!f || !y || !opts || !ws) return BF_ERR_INVALID_ARG;
    if (ms)
        for (int i = 0; i < BF_GP_TUNE_CANDIDATES; ++i) ms[i] = -1.f;
    Plan p;
    bf_status st = make_plan(planes, H, W, sigma_s, opts, &p);
    if (st != BF_OK) return st;
    int dev = 0;
    BF_CUDA(cudaGetDevice(&dev));
    const TuneKey key{dev, planes, H, W, pitch, p.spatial, p.K, p.spatial == BF_SPATIAL_FIR ? p.w : 0};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            opts->engine = it->second.engine;
            opts->fir_two_pass = it->second.fir_two_pass;
            opts->row_threads = it->second.row_threads;
            opts->fir_tile = it->second.fir_tile;
            return BF_OK;
        }
    }
    // candidates, in the order their times are reported: the recursive filter's engines, each with
    // 256- and 512-thread row-pass CTAs; the window sum fused (32-row tiles), two-pass with either
    // row-pass CTA, fused with 16- and 64-row tiles
    bf_gp_opts cand[BF_GP_TUNE_CANDIDATES];
    int nc = 0;
    if (p.spatial == BF_SPATIAL_IIR) {
        for (int e = 0; e < 4; ++e)
            for (int rt = 256; rt <= 512; rt += 256) {
                cand[nc] = *opts;
                cand[nc].engine = e;
                cand[nc++].row_threads = rt;
            }
    } else if (p.spatial == BF_SPATIAL_FIR) {
        cand[nc] = *opts;
        cand[nc].fir_two_pass = 0;
        cand[nc].fir_tile = 32;
        cand[nc++].row_threads = 0;
        for (int rt = 256; rt <= 512; rt += 256) {
            cand[nc] = *opts;
            cand[nc].fir_two_pass = 1;
            cand[nc].fir_tile = 0;
            cand[nc++].row_threads = rt;
        }
        for (int th = 16; th <= 64; th += 48) {
            cand[nc] = *opts;
            cand[nc].fir_two_pass = 0;
            cand[nc].fir_tile = th;
            cand[nc++].row_threads = 0;
        }
    } else {
        cand[nc++] = *opts;
    }
    if (reps <= 0) reps = 5;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    EventPair ev;
    BF_CUDA(cudaEventCreate(&ev.a));
    BF_CUDA(cudaEventCreate(&ev.b));
    int best = -1;
    float best_ms = 0.f;
    for (int i = 0; i < nc; ++i) {
        size_t need = 0;
        if (bf_gp_workspace_size(planes, H, W, sigma_s, &cand[i], &need) != BF_OK || need > ws_bytes) continue;
        // one untimed run; a candidate the kernels do not cover is skipped
        if (bf_gp_forward(f, y, planes, H, W, pitch, sigma_s, sigma_r, &cand[i], ws, ws_bytes, stream) != BF_OK)
            continue;
        BF_CUDA(cudaEventRecord(ev.a, s));
        for (int r = 0; r < reps; ++r) {
            st = bf_gp_forward(f, y, planes, H, W, pitch, sigma_s, sigma_r, &cand[i], ws, ws_bytes, stream);
            if (st != BF_OK) return st;
        }
        BF_CUDA(cudaEventRecord(ev.b, s));
        BF_CUDA(cudaEventSynchronize(ev.b));
        float t = 0.f;
        BF_CUDA(cudaEventElapsedTime(&t, ev.a, ev.b));
        t /= (float)reps;
        if (ms) ms[i] = t;
        if (best < 0 || t < best_ms) {
            best = i;
            best_ms = t;
        }
    }
    if (best < 0) return BF_ERR_UNSUPPORTED;
    opts->engine = cand[best].engine;
    opts->fir_two_pass = cand[best].fir_two_pass;
    opts->row_threads = cand[best].row_threads;
    opts->fir_tile = cand[best].fir_tile;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune[key] = *opts;
    return BF_OK;
}

void bf_gp_autotune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune.clear();
}

bf_status bf_gp_batched_plan_tune(bf_gp_plan *plan, void *ws, size_t ws_bytes, void *stream, int reps)
{
    if (!plan || !ws) return BF_ERR_INVALID_ARG;
    if (ws != plan->uploaded_ws || ws_bytes < plan->total) return BF_ERR_WORKSPACE;
    char *wsb = static_cast<char *>(ws);
    for (int i = 0; i < plan->n; ++i) {
        const bf_gp_plane &q = plan->specs[i];
        bf_gp_opts o = plan->base;
        o.order = q.order;
        o.spatial = BF_SPATIAL_IIR;
        bf_status st = bf_gp_autotune(q.f, q.y, 1, q.H, q.W, q.pitch, q.sigma_s, q.sigma_r, &o,
                                      wsb + plan->off_planes + plan->sub_off[i], plan->sub_bytes[i], stream, reps,
                                      nullptr);
        if (st != BF_OK) return st;
        plan->engine[i] = o.engine;
        plan->row_threads[i] = o.row_threads;
    }
    return BF_OK;
}

bf_status bf_gp_batched_plan_engines(const bf_gp_plan *plan, int *engines)
{
    if (!plan || !engines) return BF_ERR_INVALID_ARG;
    for (int i = 0; i < plan->n; ++i) engines[i] = plan->engine[i];
    return BF_OK;
}

}  // extern "C"
