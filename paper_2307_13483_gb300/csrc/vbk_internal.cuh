// Internal declarations of the vibronic-continuum Krylov library (sm_103a).
//
// Data layout in HBM (all per-system vectors contiguous, system-major):
//   vector of one system : [d][n_1]...[n_M]  (d slowest, last mode fastest), N entries
//   batch of vectors     : [system][N]        complex (float2 or double2)
//   energy tables        : [energy][N]        the diagonal of A(E) for each distinct energy
//   block factors        : [energy][row c][k = 0..p][block]  (block index fastest)
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/vbk.h"
#include "vbk_erfcx_table.h"
#include "vbk_dfmath.cuh"

#define MAXM VBK_MAX_MODES
#define MAXS VBK_MAX_STATES
#define MAXCH VBK_MAX_CHANNELS
#define PMAX 16    // widest band handled by the thread-per-block LDL^T kernels
#define PWMAX 160  // widest band handled by the cooperative (one CTA / one warp per block) LDL^T kernels
#define MAXPAIR 20  // pair transforms of q-dependent channels (a wave couples to at most MAXS states)
#define MAXSP 64    // polynomial points of all q-dependent channels

// ------------------------------------------------------------------------------- complex
template <class R> struct cx_t;
template <> struct cx_t<float> { typedef float2 T; };
template <> struct cx_t<double> { typedef double2 T; };
template <class R> using cx = typename cx_t<R>::T;

template <class R> __host__ __device__ __forceinline__ cx<R> mkc(R a, R b) {
    cx<R> z;
    z.x = a;
    z.y = b;
    return z;
}
template <class R> __host__ __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return mkc<R>(a.x + b.x, a.y + b.y); }
template <class R> __host__ __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return mkc<R>(a.x - b.x, a.y - b.y); }
template <class R> __host__ __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
    return mkc<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class R> __host__ __device__ __forceinline__ cx<R> cscale(cx<R> a, R s) { return mkc<R>(a.x * s, a.y * s); }
// conj(a) * b
template <class R> __host__ __device__ __forceinline__ cx<R> cconjmul(cx<R> a, cx<R> b) {
    return mkc<R>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc + a*b
template <class R> __host__ __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> acc) {
    return mkc<R>(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
template <class R> __host__ __device__ __forceinline__ cx<R> cdiv(cx<R> a, cx<R> b) {
    R den = b.x * b.x + b.y * b.y;
    return mkc<R>((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
template <class R> __host__ __device__ __forceinline__ R cabs2(cx<R> a) { return a.x * a.x + a.y * a.y; }

__host__ __device__ __forceinline__ float2 to_f(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
template <class R> __host__ __device__ __forceinline__ cx<R> cvt_from_d(double2 a);
template <> __host__ __device__ __forceinline__ float2 cvt_from_d<float>(double2 a) { return to_f(a); }
template <> __host__ __device__ __forceinline__ double2 cvt_from_d<double>(double2 a) { return a; }
template <class R> __host__ __device__ __forceinline__ double2 cvt_to_d(cx<R> a) { return make_double2((double)a.x, (double)a.y); }

// --------------------------------------------------------------------------- model tables
// One off-diagonal point of the q-polynomial stencil: a (term, offset) pair.  For output
// element (d, nu) it contributes  -coef * prod_m tab[col[m] + n_m] * x[dp][nu + lin].
// col[m] < 0 means the term does not involve mode m (factor 1, delta 0).
struct DevEntry {
    double coef;
    int dp;
    int lin;
    int col[MAXM];
    int delta[MAXM];
};

// Exact unsigned division by an invariant divisor with a multiply and shifts (Granlund and
// Montgomery, "Division by invariant integers using multiplication", PLDI 1994): for d >= 2,
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n),
// n / d = (t + ((n - t) >> 1)) >> (l - 1); d = 1 is the identity.
struct FastDiv {
    unsigned m;
    int l;  // 0: divisor 1
    int d;
};
inline FastDiv make_fastdiv(int d) {
    FastDiv f;
    f.d = d;
    if (d <= 1) {
        f.m = 0;
        f.l = 0;
        return f;
    }
    int l = 0;
    while ((1LL << l) < d) ++l;
    f.l = l;
    f.m = (unsigned)((((unsigned long long)1 << 32) * (((unsigned long long)1 << l) - (unsigned long long)d)) /
                         (unsigned long long)d + 1ULL);
    return f;
}
__host__ __device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
    if (f.l == 0) return n;
#ifdef __CUDA_ARCH__
    const unsigned t = __umulhi(f.m, n);
#else
    const unsigned t = (unsigned)(((unsigned long long)f.m * n) >> 32);
#endif
    return (t + ((n - t) >> 1)) >> (f.l - 1);
}

struct DevModel {
    int ns, M, Nnu, N, nmu, nchan;
    FastDiv fd_nb[MAXM];  // division by n_basis[m]
    FastDiv fd_nnu;       // division by Nnu
    int nb[MAXM], stride[MAXM];
    double omega[MAXM];
    int ebeg[MAXS + 1];  // off-diagonal stencil points of output state d: [ebeg[d], ebeg[d+1])
    int lmin[MAXS], lmax[MAXS];  // range of the in-plane offsets `lin` of the points of state d (with 0)
    int dbeg[MAXS + 1];  // diagonal parts (delta = 0, dp = d) of the terms of state d
    const DevEntry* ent;
    const DevEntry* dent;
    const double* enu;  // E_nu = sum_m omega_m (n_m + 1/2), per nu
    const double* u0;   // delta = 0 part of U_dd(nu) (the diagonal terms), per element (d, nu)
    const double* tab64;
    const float* tab32;
    int ntab;  // entries of tab64 / tab32
    // coefficient columns of the off-diagonal stencil points: pc[k][nu] = coef_k * prod_m
    // (q_m^pow)_{n_m, n_m + delta_m}, zero where the neighbour leaves the basis (energy-independent)
    const double* pc64;
    const float* pc32;
    const float2* pcs;  // the same columns as double-float pairs (hi = (float)c, lo = (float)(c - hi))
    // the same stencil for the one-block-per-system kernel, points of state d grouped by their
    // primary mode m (rbeg[d] + sum of rcnt[d][< m] ...): per point a descriptor (x: byte offset
    // of its coefficient row in rct, y: byte offset (8 ((dp - d) Nnu + lin)) of the neighbour,
    // z: tab32 column of a secondary mode or -1, w: that mode) and the row
    // rct[x / 8 + n] = -(coef (q^k)_{n, n + delta}) twice (a packed pair; zero where the neighbour
    // leaves the basis), n the primary-mode index
    const int4* rdesc;
    const float2* rct;
    const float2* rctd;  // the same rows as double-float pairs (hi, lo) of +coef (q^k)_{n, n + delta}
    const double* rct64;  // the same rows in FP64, -coef (q^k)_{n, n + delta} (one value per n)
    // the same points for the windowed matvec (in rdesc order): x = byte offset of the point's
    // row in rct, y = in-plane offset lin, z = tab32 column of a secondary mode or -1,
    // w = secondary mode | (neighbour state dp << 8)
    const int4* wdesc;
    int rsec;            // 1 if some point involves a secondary mode
    int nrct;
    int rbeg[MAXS + 1];
    int rcnt[MAXS][MAXM];
    int rhalo;   // largest distance a neighbour index falls outside [0, N)
    int rok;     // 1 if no point involves more than two modes and no state more than 64 points
    // double-float forms for the FP32 refinement path's energy tables (vbk_dfmath.cuh): the
    // interpolants of Dawson's integral and erfcx, the Taylor coefficients of Dawson's
    // integral, the delta = 0 part of U_dd per element, and per channel (a, b, sqrt b,
    // 1 / sqrt b, 1 / b)
    const float2* dawson_df;
    const float2* erfcx_df;
    const float2* taylor_df;
    const float2* u0df;
    float2 ch_df[MAXCH][5];
    int ch_d[MAXCH], ch_mu[MAXCH], ch_l[MAXCH];
    double ch_a[MAXCH], ch_b[MAXCH], ch_sb[MAXCH];  // ch_sb = sqrt(b)
    double ch_isb[MAXCH], ch_ib[MAXCH];            // 1 / sqrt(b), 1 / b
    int mu_d[MAXCH];  // discrete state coupled to partial wave mu (-1: none, or a q-dependent wave)
    // q-dependent continuum coupling (Sec. II.C, Eq. FE).  The channels of a partial wave that
    // couples to several states or through a polynomial P_c(q) are "sandwich" channels
    // j = 0..nsc-1: instead of a diagonal term they act as  F x = sum_j P_j w_j  with
    // w_j = sum_j' g_(j,j') P_j' x_(d_j'),  g_(j,j')(nu) = F[f_j f_j'](E - E_nu) for j, j' of one wave.
    int ch_sw[MAXCH];  // 1 if channel c is a sandwich channel
    int mu_sw[MAXCH];  // 1 if partial wave mu has sandwich channels
    int nsc, npair;
    int sc_ch[MAXCH], sc_d[MAXCH], sc_mu[MAXCH];
    int sc_pbeg[MAXCH + 1];     // polynomial points of sandwich channel j: [sc_pbeg[j], sc_pbeg[j + 1])
    int sc_pair[MAXCH][MAXCH];  // pair-table index of (j, j') of one wave (symmetric), -1 otherwise
    int pr_l[MAXPAIR];
    // pair transform constants: a = sqrt(a_j a_j'), b = (b_j + b_j') / 2, sqrt(b), 1 / sqrt(b), 1 / b
    double pr_a[MAXPAIR], pr_b[MAXPAIR], pr_sb[MAXPAIR], pr_isb[MAXPAIR], pr_ib[MAXPAIR];
    int sp_lin[MAXSP];  // in-plane offset of polynomial point k (the offsets of one channel are distinct)
    // spc[k][nu] = (P_j)_{nu, nu + lin_k} for point k of channel j, zero where nu + lin_k leaves the
    // basis; P_j is symmetric, so the same column gives (P_j)_{nu + lin_k, nu}
    const double* spc64;
    const float* spc32;
    // per-call buffers, set on a solver's or operator's own copy of the model (null in the model)
    double2* sg64;   // g[e][pair][nu]
    float2* sg32;
    double2* sfd64;  // diagonal of the sandwich operator [e][N] (it is part of the diagonal tables)
    float2* sfd32;
    double2* sw64;   // w[list slot][j][nu]
    float2* sw32;
};

// Host copy of a term, channel etc.
struct HostEntry {
    int d;       // output state
    int term;    // index of the generating term (for gradients)
    int mirror;  // 1 if this point comes from the transposed block of an off-diagonal term
    DevEntry e;
    double w = 1.0;  // d(point coefficient) / d(term coefficient): 1/2 for the halves of (T + T^T)/2
};

struct KTimer {
    std::string name;
    long long launches = 0;
    double ms = 0.0;
};

struct vbk_model {
    vbk_model_desc desc;  // with pointers into the vectors below
    std::vector<vbk_term> terms;
    std::vector<vbk_channel> chans;
    std::vector<vbk_cterm> cterms;
    void* dev_mem2 = nullptr;  // coefficient columns of the coupling polynomials (q-dependent channels)
    void* dev_mem3 = nullptr;  // double-float tables of the energy diagonal (vbk_dfmath.cuh)
    std::vector<std::vector<int>> sp_delta;  // per polynomial point of a sandwich channel: offset per mode
    int M = 0, ns = 0, Nnu = 0, N = 0, nmu = 0;
    int nb[MAXM] = {0}, stride[MAXM] = {0};
    std::vector<double> tab;          // per-(mode, power, offset) columns of (q^k)_{n, n+delta}
    std::vector<HostEntry> offd;      // off-diagonal stencil points, grouped by d
    std::vector<HostEntry> diagp;     // diagonal parts, grouped by d
    std::vector<std::vector<int>> colbase;  // colbase[m][k] = start of power k columns in tab
    DevModel dm{};
    void* dev_mem = nullptr;  // one allocation holding entries and tables
    // bookkeeping of the last solve
    std::vector<KTimer> timers;
    long long launches = 0;
    int device = 0;
    cudaStream_t cap_stream = nullptr;  // library-owned stream used only to capture CUDA graphs
    int mv_variant[2] = {-1, -1};       // autotuned matvec variant per precision (FP32, FP64); -1: untuned
    int op_timing = 0;                  // 1: vbk_matvec / vbk_precond_apply record per-kernel timings
    cudaMemPool_t pool = nullptr;       // library-owned stream-ordered pool (keeps its memory between calls)
    void* hpin = nullptr;               // library-owned pinned host staging buffer (grown on demand)
    size_t hpin_bytes = 0;
};

// The model's pinned staging buffer with at least `bytes` bytes (callers have synchronised every
// copy that used the previous contents before they return).
inline void* vbk_pinned(vbk_model* m, size_t bytes) {
    if (m->hpin_bytes < bytes) {
        if (m->hpin) cudaFreeHost(m->hpin);
        m->hpin = nullptr;
        m->hpin_bytes = 0;
        const size_t want = bytes < (size_t)65536 ? (size_t)65536 : bytes * 2;
        if (cudaMallocHost(&m->hpin, want) != cudaSuccess) {
            cudaGetLastError();
            m->hpin = nullptr;
            return nullptr;
        }
        m->hpin_bytes = want;
    }
    return m->hpin;
}

// --------------------------------------------------------------------------- level shift
// Dawson's integral D(x) = exp(-x^2) int_0^x exp(t^2) dt, odd in x.  |x| < 1/2: Taylor series
// D(x) = x sum_k (-2 x^2)^k / (2k + 1)!!, 14 terms (truncation below 1e-16); 1/2 <= |x| < 16:
// piecewise degree-12 polynomials on intervals of width 1/2 (interpolation at Chebyshev points,
// coefficients computed in 40-digit arithmetic by gen_erfcx_table.py; relative error ~3e-15);
// from 16: the asymptotic series D(x) = 1/(2x) sum_k (2k - 1)!! / (2 x^2)^k, 9 terms.
static __device__ const double vbk_dawson_c_dev[VBK_ERFCX_NINT * (VBK_ERFCX_DEG + 1)] = {VBK_DAWSON_COEFFS};
static const double vbk_dawson_c_host[VBK_ERFCX_NINT * (VBK_ERFCX_DEG + 1)] = {VBK_DAWSON_COEFFS};
__host__ __device__ inline double vbk_dawson(double x) {
    const double ax = fabs(x);
    double r;
    if (ax < 0.5) {
        const double u = ax * ax;
        // (-2)^k / (2k + 1)!!, k = 0..13 (quotients of exact constants, folded at compile time)
        const double cs[14] = {1.0,
                               -2.0 / 3.0,
                               4.0 / 15.0,
                               -8.0 / 105.0,
                               16.0 / 945.0,
                               -32.0 / 10395.0,
                               64.0 / 135135.0,
                               -128.0 / 2027025.0,
                               256.0 / 34459425.0,
                               -512.0 / 654729075.0,
                               1024.0 / 13749310575.0,
                               -2048.0 / 316234143225.0,
                               4096.0 / 7905853580625.0,
                               -8192.0 / 213458046676875.0};
        r = cs[13];
        for (int k = 12; k >= 0; --k) r = fma(r, u, cs[k]);
        r *= ax;
    } else if (ax < 0.5 * VBK_ERFCX_NINT) {
#ifdef __CUDA_ARCH__
        const double* C = vbk_dawson_c_dev;
#else
        const double* C = vbk_dawson_c_host;
#endif
        const int k = (int)(2.0 * ax);
        const double t = 4.0 * ax - (double)(2 * k + 1);
        const double* c = C + k * (VBK_ERFCX_DEG + 1);
        r = c[VBK_ERFCX_DEG];
        for (int p = VBK_ERFCX_DEG - 1; p >= 0; --p) r = fma(r, t, c[p]);
    } else {
        const double u = 0.5 / (ax * ax);
        double sum = 1.0, term = 1.0;
        for (int k = 1; k <= 8; ++k) {
            term *= (2.0 * k - 1.0) * u;
            sum += term;
        }
        r = 0.5 / ax * sum;
    }
    return x < 0 ? -r : r;
}

// erfcx(y) = exp(y^2) erfc(y), y >= 0.  Below 16: piecewise degree-12 polynomials on intervals
// of width 1/2 (interpolation at Chebyshev points of each interval, coefficients computed in
// 40-digit arithmetic by gen_erfcx_table.py; relative error ~1e-15).  From 16: the asymptotic
// series erfcx(y) = 1 / (y sqrt(pi)) sum_k (-1)^k (2k - 1)!! / (2 y^2)^k, 9 terms (the first
// omitted term is below 1e-16 there).
static __device__ const double vbk_erfcx_c_dev[VBK_ERFCX_NINT * (VBK_ERFCX_DEG + 1)] = {VBK_ERFCX_COEFFS};
static const double vbk_erfcx_c_host[VBK_ERFCX_NINT * (VBK_ERFCX_DEG + 1)] = {VBK_ERFCX_COEFFS};
__host__ __device__ inline double vbk_erfcx(double y) {
    if (y < 0.5 * VBK_ERFCX_NINT) {
#ifdef __CUDA_ARCH__
        const double* C = vbk_erfcx_c_dev;
#else
        const double* C = vbk_erfcx_c_host;
#endif
        const int k = y > 0.0 ? (int)(2.0 * y) : 0;
        const double t = 4.0 * y - (double)(2 * k + 1);
        const double* c = C + k * (VBK_ERFCX_DEG + 1);
        double r = c[VBK_ERFCX_DEG];
        for (int p = VBK_ERFCX_DEG - 1; p >= 0; --p) r = fma(r, t, c[p]);
        return r;
    }
    const double u = 0.5 / (y * y);
    double s = 1.0, term = 1.0;
    for (int k = 1; k <= 8; ++k) {
        term *= -(2.0 * k - 1.0) * u;
        s += term;
    }
    return 0.56418958354775628 / y * s;
}

// F[f](eps) for f(x) = (a / 2 pi) x^(l+1/2) exp(-b x), x > 0 (Eq. IntF with the widths of
// Sec. II.B):  (a/2pi) [ P_l(eps) - i pi eps^(l+1/2) exp(-b eps) theta(eps) ]  with
//   P_l = -Gamma(l+1/2) b^-(l+1/2) + eps P_(l-1),
//   eps P_(-1) = 2 sqrt(pi eps) D(sqrt(b eps))  (eps > 0),  pi sqrt(-eps) erfcx(sqrt(-b eps))
//   (eps < 0), 0 (eps = 0).
__host__ __device__ inline double2 vbk_level_shift_eval(double eps, double a, double b, int l) {
    const double PI = 3.14159265358979323846;
    double t;
    if (eps > 0.0)
        t = 2.0 * sqrt(PI * eps) * vbk_dawson(sqrt(b * eps));
    else if (eps < 0.0)
        t = PI * sqrt(-eps) * vbk_erfcx(sqrt(-b * eps));
    else
        t = 0.0;
    double g = 1.7724538509055160;  // Gamma(1/2) = sqrt(pi)
    double bp = sqrt(b);            // b^(k+1/2) for k = 0
    double p = -g / bp + t;
    for (int k = 1; k <= l; ++k) {
        g *= (k - 0.5);  // Gamma(k + 1/2)
        bp *= b;
        p = -g / bp + eps * p;
    }
    double im = 0.0;
    if (eps > 0.0) im = -0.5 * a * pow(eps, l + 0.5) * exp(-b * eps);
    return make_double2(a / (2.0 * PI) * p, im);
}

// The same transform from precomputed channel constants sb = sqrt(b), isb = 1 / sqrt(b),
// ib = 1 / b: one square root and no division per evaluation (sqrt(b |eps|) = sb sqrt(|eps|),
// Gamma(k + 1/2) b^-(k+1/2) built up by multiplications).
__host__ __device__ inline double2 vbk_level_shift_core(double eps, double a, double b, double sb, double isb, double ib,
                                                        int l) {
    const double PI = 3.14159265358979323846;
    const double SQRT_PI = 1.7724538509055160;
    const double sq = sqrt(fabs(eps));
    double t;
    if (eps > 0.0)
        t = 2.0 * SQRT_PI * sq * vbk_dawson(sb * sq);
    else if (eps < 0.0)
        t = PI * sq * vbk_erfcx(sb * sq);
    else
        t = 0.0;
    double g = SQRT_PI;  // Gamma(k + 1/2), k = 0
    double ibp = isb;    // b^-(k+1/2)
    double p = t - g * ibp;
    for (int k = 1; k <= l; ++k) {
        g *= (k - 0.5);
        ibp *= ib;
        p = eps * p - g * ibp;
    }
    double im = 0.0;
    if (eps > 0.0) {
        double el = sq;  // eps^(l+1/2)
        for (int k = 0; k < l; ++k) el *= eps;
        im = -0.5 * a * el * exp(-b * eps);
    }
    return make_double2(a * (0.5 / PI) * p, im);
}
__host__ __device__ inline double2 vbk_level_shift_eval_sb(double eps, double a, double b, double sb, int l) {
    return vbk_level_shift_core(eps, a, b, sb, 1.0 / sb, 1.0 / b, l);
}

// The double-float tables of the level shift built on the host from the FP64 ones: Dawson
// interpolants, erfcx interpolants (VBK_ERFCX_NINT x 13 pairs each) and Dawson's Taylor
// coefficients (14 pairs).
inline void vbk_df_tables(std::vector<float2>* dawson, std::vector<float2>* erfcx, std::vector<float2>* taylor) {
    const int n = VBK_ERFCX_NINT * (VBK_ERFCX_DEG + 1);
    dawson->resize(n);
    erfcx->resize(n);
    for (int k = 0; k < n; ++k) {
        const dflt a = dd_from(vbk_dawson_c_host[k]), b = dd_from(vbk_erfcx_c_host[k]);
        (*dawson)[k] = make_float2(a.h, a.l);
        (*erfcx)[k] = make_float2(b.h, b.l);
    }
    taylor->resize(14);
    double c = 1.0, dfact = 1.0;  // (-2)^k / (2k + 1)!!
    for (int k = 0; k < 14; ++k) {
        if (k > 0) {
            c *= -2.0;
            dfact *= (double)(2 * k + 1);
        }
        const dflt t = dd_from(c / dfact);
        (*taylor)[k] = make_float2(t.h, t.l);
    }
}

// f(eps) = sqrt(Gamma(eps) / 2 pi), zero for eps <= 0 (reading: closed channels do not couple)
__host__ __device__ inline double vbk_amplitude(double eps, double a, double b, int l) {
    if (!(eps > 0.0)) return 0.0;
    const double PI = 3.14159265358979323846;
    return sqrt(a * pow(eps, l + 0.5) * exp(-b * eps) / (2.0 * PI));
}

// --------------------------------------------------------------------------- helpers
// Stream-ordered allocation from the model's own pool: workspace freed at the end of a call stays
// reserved in the pool (release threshold: unlimited), so repeated solves do not map memory again.
inline cudaError_t vbk_alloc(const vbk_model* m, void** p, size_t bytes, cudaStream_t st) {
    return m->pool ? cudaMallocFromPoolAsync(p, bytes, m->pool, st) : cudaMallocAsync(p, bytes, st);
}
void vbk_set_error(const std::string& msg);
int vbk_cuda_fail(cudaError_t e, const char* what);
#define VBK_CUDA(call)                                             \
    do {                                                           \
        cudaError_t e__ = (call);                                  \
        if (e__ != cudaSuccess) return vbk_cuda_fail(e__, #call);  \
    } while (0)

// Per-system solver state (device).
struct SysState {
    double bnorm;    // ||b|| (FP64)
    double rnorm;    // ||b - A x|| of the last FP64 residual
    double scale;    // ||r|| used to scale the inner right-hand side
    double inv_scale;  // 1 / scale (computed once per refinement step)
    double target;   // inner stopping threshold relative to the (unit) inner rhs
    double pscale;   // scale of the previous inner solve (0: none yet)
    double2 rho;     // COCG r^T z
    double2 alpha;
    double2 beta;
    double inres;    // inner residual norm
    int status;
    int outer;       // 1 while the system still needs work
    int inner;       // 1 while the inner solve runs
    int iters;       // Krylov iterations
    int refines;     // FP64 residuals after the first
    int j;           // GMRES: steps in the current cycle
    int cycle_iters; // iterations in the current inner solve
    int last_cycle;  // iterations of the previous inner solve (orders the next launch)
    int icap;        // iteration count at which the current inner solve stops (<= max_iter)
};

// Internal per-system status (never returned to callers): a VBK_MIXED refinement step that
// lowered the FP64 residual by less than 10%; such systems are solved again in FP64.
#define VBK_SYS_STALLED 6

// Fused mixed-precision solve on thread-block clusters (vbk_cluster.cu): one cluster of n_s CTAs
// per system runs the whole refinement (FP32 COCG with the point preconditioner or none, the
// double-float residual, the checks) and writes psi in FP64.
struct ClArgs {
    int nsys = 0, pmode = 0, max_refine = 0, max_iter = 0, inner_cap = 0, stall_check = 0;
    int halo = 0, nrow = 0, npt = 0;  // set by vbk_cluster_plan
    double tol = 0.0, inner_tol = 0.0;
    int* counter = nullptr;             // zero before the launch
    const int* sys_e = nullptr;         // energy index of each system
    const float2* diag32 = nullptr;     // [energy][N] FP32 diagonal of A
    const float4* diagdf = nullptr;     // [energy][N] double-float diagonal of A
    const double2* b64 = nullptr;       // [system][N]
    const double* bn2 = nullptr;        // ||b||^2 per system, or null
    float4* xs = nullptr;               // [system][N] double-float solution, zero before the launch
    double2* psi = nullptr;             // [system][N] FP64 solution (written)
    SysState* st = nullptr;             // per-system record (written)
    // quad loops of the one-CTA solve: fast divisors by the digit radices (n_s, nb_0 .. nb_{M-3},
    // nb_{M-2} / 4, nb_{M-1}) of a quad index (entries M.. unused) and the digits of the thread
    // stride, set on the host (kernel parameters: no registers held)
    FastDiv qfd[MAXM] = {};
    int qinc[MAXM] = {}, qincd = 0;
};
bool vbk_cluster_plan(const DevModel& md, ClArgs* a, size_t* smem);
int vbk_cluster_prepare(const DevModel& md, const ClArgs& a, size_t smem, int* max_clusters);
cudaError_t vbk_cluster_launch(const DevModel& md, const ClArgs& a, size_t smem, int nclusters, cudaStream_t st);

// Streaming batched matvec (vbk_stream.cu): persistent CTAs over tiles of S systems x TR rows of
// mode 0 (all states), the x windows and diagonal rows of each tile brought into a ring of nst
// shared-memory stages by bulk asynchronous copies.  Offered for models with n_s N_nu / n_0 <= 640
// and at most two modes per stencil point; partial sums (red != 0) go to part[system][strip].
constexpr int ST_MAXSTAGE = 4;
struct StreamPlan {
    int S = 1, RG = 1, TR = 1, nst = 2;         // systems per tile, row groups, rows per tile, stages
    int ndg = 1;                                // diagonal buffers per stage (energies staged per tile)
    int R = 0, nstrip = 0, lo = 0, W = 0;  // row length, strips, window start offset and length
    int npg = 0, np = 0;  // stencil points per state (padded); table columns
    int threads = 0;
    unsigned stage_bytes = 0, win_bytes = 0;  // bytes of one stage; of which the x windows
    size_t smem = 0;                          // dynamic shared memory of a CTA
    unsigned long long delay_ns = 0;          // test hook: the producers hold their first copies back
};
int vbk_stream_nconfig();
bool vbk_stream_plan(const DevModel& md, int cfg, size_t c, StreamPlan* p);
cudaError_t vbk_stream_matvec(const DevModel& md, const StreamPlan& p, const int* sys_e, const int* list, const int* act,
                              int nlist, const void* diag, const void* x, long long xs, void* y, long long ys,
                              const double2* b, double2* part, int red, bool fp32, cudaStream_t st);
int vbk_stream_prepare(const DevModel& md, bool fp32);  // shared-memory opt-in (outside stream capture)
unsigned vbk_stream_fault_take();
int vbk_debug_stream_delay_impl(int ms);

// Internal solve over an explicit list of systems with dense FP64 right-hand sides.
struct SolveJob {
    int nsys = 0;
    int nE = 0;
    std::vector<double> E;      // distinct total energies
    std::vector<int> sys_e;     // energy index of each system
    const double2* b64 = nullptr;  // device [nsys][N]
    double2* x64 = nullptr;        // device [nsys][N] (output)
    const double* bnorm2 = nullptr;  // device [nsys] ||b||^2 when the caller built b, else computed from b
};
int vbk_solve_job(vbk_model* m, const SolveJob& job, const vbk_opts& o, vbk_stats* st, cudaStream_t stream);

// Block-preconditioner plan (Sec. III.B)
struct BlockPlan {
    int span = 0;
    int L = 1;      // chain (block) length
    int nblk = 0;   // blocks per energy
    int p = 0;      // half bandwidth in chain order
    bool wide = false;  // p > PMAX: level-blocked factor (levels of S chain positions, K levels)
    int S = 0, K = 0;
    std::vector<int> ent_dc;  // per off-diagonal stencil point: chain offset (0 = outside block)
    // entries of the sandwich operator inside a block (q-dependent couplings, Eq. FE): for row
    // state d, points k of P_j (d_j = d) and k2 of P_j' (j' of the same wave), the entry
    // (d, nu) -> (d_j', nu + lin_k + lin_k2) receives spc[k][nu] g_(j,j')(nu + lin_k) spc[k2][nu + lin_k];
    // five ints each: d, k, k2, pair, chain offset (nonzero)
    std::vector<int> sw_combo;
};
int vbk_make_block_plan(const vbk_model* m, int span, BlockPlan* plan);

// launch helpers implemented in vbk_kernels.cu
struct Launch;

// y = A x (op 0) or z = B^-1 r (op 1) outside a solve (implemented in vbk_solver.cu)
int vbk_operator_run(vbk_model* m, int op, int nE, const double* E, int nvec, int span, const double2* x, double2* y,
                     int precision, cudaStream_t st, int variant = -1);
