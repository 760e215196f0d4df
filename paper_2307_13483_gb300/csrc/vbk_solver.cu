// Batched preconditioned Krylov solver for (E - H_ef) psi = Phi on sm_103a.
//
// Hot path of Sec. III: the matrix-free matvec (diagonal energy/level-shift factors plus the
// q-polynomial ladder stencils), block-diagonal preconditioners factored as L D L^T
// (Sec. III.B), restarted GMRES with CGS2 Arnoldi and an FP64 Givens least-squares problem,
// and COCG with the bilinear form a^T b (Sec. III.A).  Every (energy, initial state, partial
// wave) system of a batch is advanced by the same grid-wide kernels; a per-system mask
// retires converged systems.  The Krylov iterations run in complex FP32 or FP64 inside an FP64
// iterative-refinement loop whose residual b - A x is always evaluated in FP64.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "vbk_internal.cuh"
#include "vbk_device.cuh"

namespace {

constexpr int TPB = 256;       // threads per block, element-wise kernels
constexpr int VEPT = 4;        // elements per thread in the basis-vector kernels
constexpr int VCHUNK = TPB * VEPT;
constexpr int BTPB = 64;       // threads per block, block-preconditioner kernels
// narrowing / widening helpers used by the stand-alone entry points
__global__ void k_inner_rhs_plain(long long n, const double2* __restrict__ a, float2* __restrict__ b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = to_f(a[i]);
}
__global__ void k_widen(long long n, const float2* __restrict__ a, double2* __restrict__ b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = to_d(a[i]);
}

// ----------------------------------------------------------------------------- reductions
__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Sum over the block; the result is valid in thread 0.  `sh` holds >= 32 double2.
__device__ __forceinline__ double2 block_sum2(double2 v, double2* sh) {
    v = warp_sum2(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? sh[lane] : make_double2(0.0, 0.0);
        r = warp_sum2(r);
    }
    return r;
}


// Systems a launch covers: blockIdx.y indexes `list` (compacted active systems) when given,
// else the system itself; `act` masks systems that retired after the list was built.
struct Sel {
    const int* list;
    const int* act;
};
__device__ __forceinline__ int sel_sys(const Sel& q) { return q.list ? q.list[blockIdx.y] : (int)blockIdx.y; }

// Sum over the block in the kernel's own precision (GB300 executes FP64 at a small fraction of
// the FP32 rate, so FP32 kernels reduce in FP32); widened to double in thread 0 only.
template <class R> __device__ __forceinline__ cx<R> warp_sum_c(cx<R> v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}
template <class R> __device__ __forceinline__ double2 block_sum_c(cx<R> v, cx<R>* sh) {
    v = warp_sum_c<R>(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    cx<R> r = mkc<R>(0, 0);
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? sh[lane] : mkc<R>(0, 0);
        r = warp_sum_c<R>(r);
    }
    return cvt_to_d<R>(r);
}

template <class R> __device__ __forceinline__ const R* tabp(const DevModel& md);
template <> __device__ __forceinline__ const float* tabp<float>(const DevModel& md) { return md.tab32; }
template <> __device__ __forceinline__ const double* tabp<double>(const DevModel& md) { return md.tab64; }


// Coefficient of one stencil point at oscillator coordinates n; false if the neighbour lies
// outside the truncated basis (the table holds zero there as well).
template <class R, int M>
__device__ __forceinline__ bool point_coef(const DevEntry& en, const int (&n)[MAXM], const DevModel& md, const R* tab,
                                           R& c) {
    R v = (R)en.coef;
    bool ok = true;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int col = en.col[m];
        if (col >= 0) {
            const int nn = n[m] + en.delta[m];
            ok = ok && nn >= 0 && nn < md.nb[m];
            v *= tab[col + n[m]];
        }
    }
    c = v;
    return ok;
}

// ------------------------------------------------------------------------ level-shift table
// diag[e][i] = E_e - E_nu - (delta = 0 part of U_dd)(nu) - sum_{channels of d} F(E_e - E_nu)
// (Eqs. H_ef, Amatrix; Sec. III "energy-dependent diagonal factors"), FP64, with an optional
// FP32 copy for the inner iterations.
template <int M>
__global__ void k_diag_table(DevModel md, int nE, const double* __restrict__ E, double2* __restrict__ d64,
                             float2* __restrict__ d32, float2* __restrict__ dinv32, float4* __restrict__ dsp,
                             int* __restrict__ zpiv) {
    const int e = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;  // grid: elements x energies
    if (i >= md.N) return;
    const long long t = (long long)e * md.N + i;
    const int d = (int)fdiv((unsigned)i, md.fd_nnu), nu = i - d * md.Nnu;
    // E_nu and the delta = 0 part of U_dd are energy-independent: tabulated at model build
    const double eps = E[e] - md.enu[nu];
    double re = eps - md.u0[i], im = 0.0;
    for (int c = 0; c < md.nchan; ++c) {
        if (md.ch_d[c] != d || md.ch_sw[c]) continue;
        const double2 F =
            vbk_level_shift_core(eps, md.ch_a[c], md.ch_b[c], md.ch_sb[c], md.ch_isb[c], md.ch_ib[c], md.ch_l[c]);
        re -= F.x;
        im -= F.y;
    }
    if (md.nsc) {
        // diagonal of the sandwich operator (Eq. FE): sum_j sum_k (P_j)_{nu, nu+lin_k}^2 g_(j,j)(nu + lin_k),
        // from the pair tables written by k_sand_table; part of diag(A), added back by the matvec
        double fr = 0.0, fi = 0.0;
        for (int j = 0; j < md.nsc; ++j) {
            if (md.sc_d[j] != d) continue;
            const double2* g = md.sg64 + ((long long)e * md.npair + md.sc_pair[j][j]) * md.Nnu;
            for (int k = md.sc_pbeg[j]; k < md.sc_pbeg[j + 1]; ++k) {
                const double c = md.spc64[(long long)k * md.Nnu + nu];
                if (c != 0.0) {  // nonzero only where nu + lin_k lies in the basis
                    const double2 gv = g[nu + md.sp_lin[k]];
                    fr = fma(c * c, gv.x, fr);
                    fi = fma(c * c, gv.y, fi);
                }
            }
        }
        re -= fr;
        im -= fi;
        md.sfd64[t] = make_double2(fr, fi);
        if (md.sfd32) md.sfd32[t] = make_float2((float)fr, (float)fi);
    }
    if (d64) d64[t] = make_double2(re, im);
    // a zero diagonal entry is a zero pivot of the point (Jacobi) preconditioner, in FP64 or in
    // the FP32 copy the inner iterations use
    if (zpiv && ((re == 0.0 && im == 0.0) || (d32 && (float)re == 0.f && (float)im == 0.f))) zpiv[e] = 1;
    if (dsp) {  // double-float pair (hi, lo) of the FP64 value for the double-float residual
        const float hr = (float)re, hi = (float)im;
        dsp[t] = make_float4(hr, hi, (float)(re - (double)hr), (float)(im - (double)hi));
    }
    if (d32) {
        const float2 f = make_float2((float)re, (float)im);
        d32[t] = f;
        if (dinv32) {  // 1 / diag in FP32 for the Jacobi step of the FP32 iterations
            const float den = f.x * f.x + f.y * f.y;
            dinv32[t] = make_float2(f.x / den, -f.y / den);
        }
    }
}

// Energy tables of the FP32 refinement path, in double-float arithmetic on the FP32 pipes
// (vbk_dfmath.cuh): diag[e][d, nu] = E_e - E_nu - U_dd^(delta=0)(nu) - sum_ch F[Gamma/2pi](E_e - E_nu)
// as the split (re hi, im hi, re lo, im lo), its FP32 rounding and the FP32 reciprocal.  The
// only FP64 arithmetic per element is E_e - E_nu and its split (models with q-dependent
// couplings take the FP64 kernel above).  Grid: elements x energies.
__global__ void __launch_bounds__(TPB) k_diag_table_df(DevModel md, int nE, const double* __restrict__ E,
                                                      float2* __restrict__ d32, float2* __restrict__ dinv32,
                                                      float4* __restrict__ dsp, int* __restrict__ zpiv) {
    const int e = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= md.N) return;
    const long long t = (long long)e * md.N + i;
    const int d = (int)fdiv((unsigned)i, md.fd_nnu), nu = i - d * md.Nnu;
    const double epsd = E[e] - md.enu[nu];
    const float eh = (float)epsd;
    const dflt eps = dfv(eh, (float)(epsd - (double)eh));
    const float2 u0 = md.u0df[i];
    dflt re = dd_sub(eps, dfv(u0.x, u0.y)), im = dfv(0.f);
    const DfLevelShift T{md.dawson_df, md.erfcx_df, md.taylor_df, VBK_ERFCX_NINT};
    for (int c = 0; c < md.nchan; ++c) {
        if (md.ch_d[c] != d) continue;
        dflt fr, fi;
        dd_level_shift(eps, md.ch_df[c], md.ch_l[c], T, &fr, &fi);
        re = dd_sub(re, fr);
        im = dd_sub(im, fi);
    }
    dsp[t] = make_float4(re.h, im.h, re.l, im.l);
    const float2 f = make_float2(re.h, im.h);
    d32[t] = f;
    if (dinv32) {
        const float den = f.x * f.x + f.y * f.y;
        dinv32[t] = make_float2(f.x / den, -f.y / den);
    }
    if (zpiv && f.x == 0.f && f.y == 0.f) zpiv[e] = 1;  // a zero pivot of the point preconditioner
}

// Batched matvec y = A x (or y = b - A x): one thread owns one element of one state and applies
// its stencil to S systems.  The off-diagonal part of A is energy-independent, so the coefficient
// of every stencil point is read once per element (precomputed column, L2-resident) and reused
// for the S systems; only the diagonal table depends on the energy.  Neighbour indices are
// clamped into the vector (their coefficient is zero there).  Grid: x = (state d, chunk of TPB
// elements), y = groups of S systems of the list.  Optional partials (red = 1: x^T y,
// red = 2: ||y||^2) per (system, blockIdx.x), reduced in the kernel's precision.
constexpr int MV_MAXPTS = 256;

template <class R> __device__ __forceinline__ const R* pcp(const DevModel& md);
template <> __device__ __forceinline__ const float* pcp<float>(const DevModel& md) { return md.pc32; }
template <> __device__ __forceinline__ const double* pcp<double>(const DevModel& md) { return md.pc64; }

// --------------------------------------------------- q-dependent coupling (Sec. II.C, Eq. FE)
// g[e][p][nu] = F[f_j f_j'](E_e - E_nu) for every pair p = (j, j') of sandwich channels of one
// partial wave, in FP64 and (when requested) FP32.
__global__ void k_sand_table(DevModel md, int nE, const double* __restrict__ E) {
    const int e = blockIdx.y, nu = blockIdx.x * blockDim.x + threadIdx.x;
    if (nu >= md.Nnu) return;
    const double eps = E[e] - md.enu[nu];
    for (int p = 0; p < md.npair; ++p) {
        const double2 F = vbk_level_shift_core(eps, md.pr_a[p], md.pr_b[p], md.pr_sb[p], md.pr_isb[p], md.pr_ib[p], md.pr_l[p]);
        const long long t = ((long long)e * md.npair + p) * md.Nnu + nu;
        md.sg64[t] = F;
        if (md.sg32) md.sg32[t] = to_f(F);
    }
}

template <class R> __device__ __forceinline__ const R* spcp(const DevModel& md);
template <> __device__ __forceinline__ const float* spcp<float>(const DevModel& md) { return md.spc32; }
template <> __device__ __forceinline__ const double* spcp<double>(const DevModel& md) { return md.spc64; }
template <class R> __device__ __forceinline__ const cx<R>* sgp(const DevModel& md);
template <> __device__ __forceinline__ const float2* sgp<float>(const DevModel& md) { return md.sg32; }
template <> __device__ __forceinline__ const double2* sgp<double>(const DevModel& md) { return md.sg64; }
template <class R> __device__ __forceinline__ const cx<R>* sfdp(const DevModel& md);
template <> __device__ __forceinline__ const float2* sfdp<float>(const DevModel& md) { return md.sfd32; }
template <> __device__ __forceinline__ const double2* sfdp<double>(const DevModel& md) { return md.sfd64; }
template <class R> __device__ __forceinline__ cx<R>* swp(const DevModel& md);
template <> __device__ __forceinline__ float2* swp<float>(const DevModel& md) { return md.sw32; }
template <> __device__ __forceinline__ double2* swp<double>(const DevModel& md) { return md.sw64; }

// Inner half of the sandwich product, per system of the list (first pass of the staged stencil):
//   u_j = P_j x_(d_j)   (polynomial points of channel j),
//   w[slot][j][nu] = sum_j' g_(j,j')(nu) u_j'(nu)   over the channels j' of the same wave.
// Grid: x = chunks of TPB levels nu, y = list slots.
template <class R>
__global__ void __launch_bounds__(TPB) k_sand_w(DevModel md, const int* __restrict__ sys_e, Sel sel, int nlist,
                                               const cx<R>* __restrict__ x, long long xs) {
    const int li = blockIdx.y, nu = blockIdx.x * TPB + threadIdx.x;
    const int Nnu = md.Nnu;
    if (nu >= Nnu || li >= nlist) return;
    int s = sel.list ? sel.list[li] : li;
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const int e = sys_e[s];
    const cx<R>* xp = x + (long long)s * xs;
    const R* pc = spcp<R>(md);
    cx<R> u[MAXCH];
#pragma unroll
    for (int j = 0; j < MAXCH; ++j) {
        u[j] = mkc<R>(0, 0);
        if (j < md.nsc) {
            const cx<R>* xd = xp + (long long)md.sc_d[j] * Nnu;
            for (int k = md.sc_pbeg[j]; k < md.sc_pbeg[j + 1]; ++k) {
                const R c = __ldg(pc + (long long)k * Nnu + nu);
                if (c != (R)0) {
                    const cx<R> v = xd[nu + md.sp_lin[k]];
                    u[j].x = fma(c, v.x, u[j].x);
                    u[j].y = fma(c, v.y, u[j].y);
                }
            }
        }
    }
    const cx<R>* g = sgp<R>(md) + (long long)e * md.npair * Nnu + nu;
    cx<R>* w = swp<R>(md) + (long long)li * md.nsc * Nnu + nu;
#pragma unroll
    for (int j = 0; j < MAXCH; ++j) {
        if (j < md.nsc) {
            cx<R> acc = mkc<R>(0, 0);
#pragma unroll
            for (int j2 = 0; j2 < MAXCH; ++j2) {
                const int p = j2 < md.nsc ? md.sc_pair[j][j2] : -1;
                if (p >= 0) acc = cfma<R>(g[(long long)p * Nnu], u[j2], acc);
            }
            w[(long long)j * Nnu] = acc;
        }
    }
}

// y = A x (or b - A x) for models with sandwich channels: the stencil of k_matvec2 (one system
// per thread) plus the outer half of the sandwich product,
//   y_d -= sum_{j: d_j = d} P_j w_j  and  y_d += diag(F_s) x_d
// (the diagonal tables hold the whole diagonal of A, including that of the sandwich operator).
// Reads w of the same list slot, written by k_sand_w.  Same grid and partials as k_matvec2<R, 1>.
template <class R>
__global__ void __launch_bounds__(TPB) k_matvec_sw(DevModel md, const int* __restrict__ sys_e, Sel sel, int nlist,
                                                  const cx<R>* __restrict__ diag, const cx<R>* __restrict__ x, long long xs,
                                                  cx<R>* __restrict__ y, long long ys, const double2* __restrict__ b,
                                                  double2* __restrict__ part, int red) {
    __shared__ int offs[MV_MAXPTS];
    __shared__ cx<R> redsh[TPB / 32];
    const int nchunk = (md.Nnu + TPB - 1) / TPB;
    const int d = blockIdx.x / nchunk;
    const int nu = (blockIdx.x - d * nchunk) * TPB + threadIdx.x;
    const int N = md.N, Nnu = md.Nnu;
    const int pb = md.ebeg[d], np = min(md.ebeg[d + 1] - pb, MV_MAXPTS);
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const DevEntry& e = md.ent[pb + k];
        offs[k] = (e.dp - d) * Nnu + e.lin;
    }
    const int li = blockIdx.y;
    int s = -1;
    if (li < nlist) {
        s = sel.list ? sel.list[li] : li;
        if (s >= 0 && sel.act && !sel.act[s]) s = -1;
    }
    __syncthreads();
    const bool on = s >= 0 && nu < Nnu;
    const int i = d * Nnu + nu;
    const cx<R>* xp = x + (long long)(s < 0 ? 0 : s) * xs;
    cx<R> acc = mkc<R>(0, 0), xi = mkc<R>(0, 0);
    if (on) {
        const long long te = (long long)sys_e[s] * N + i;
        xi = xp[i];
        acc = cmul<R>(cadd<R>(diag[te], sfdp<R>(md)[te]), xi);
        const R* pc = pcp<R>(md) + (long long)pb * Nnu + nu;
        for (int k = 0; k < np; ++k) {
            const R c = __ldg(pc + (long long)k * Nnu);
            if (c != (R)0) {
                const cx<R> v = xp[min(max(i + offs[k], 0), N - 1)];
                acc.x = fma(-c, v.x, acc.x);
                acc.y = fma(-c, v.y, acc.y);
            }
        }
        const R* sp = spcp<R>(md);
        for (int j = 0; j < md.nsc; ++j) {
            if (md.sc_d[j] != d) continue;
            const cx<R>* wj = swp<R>(md) + ((long long)li * md.nsc + j) * Nnu;
            for (int k = md.sc_pbeg[j]; k < md.sc_pbeg[j + 1]; ++k) {
                const R c = __ldg(sp + (long long)k * Nnu + nu);
                if (c != (R)0) {
                    const cx<R> v = wj[nu + md.sp_lin[k]];
                    acc.x = fma(-c, v.x, acc.x);
                    acc.y = fma(-c, v.y, acc.y);
                }
            }
        }
    }
    cx<R> loc = mkc<R>(0, 0);
    if (on) {
        cx<R> out = acc;
        if (b) {
            const double2 bb = b[(long long)s * N + i];
            out = mkc<R>((R)bb.x - out.x, (R)bb.y - out.y);
        }
        y[(long long)s * ys + i] = out;
        if (red == 1) loc = cmul<R>(xi, out);
        else if (red == 2) {
            const float ox = (float)out.x, oy = (float)out.y;
            loc = mkc<R>((R)(ox * ox + oy * oy), 0);
        }
    }
    if (red) {
        const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
        const cx<R> v = warp_sum_c<R>(loc);
        if (lane == 0) redsh[wp] = v;
        __syncthreads();
        if (threadIdx.x == 0 && s >= 0) {
            cx<R> tot = mkc<R>(0, 0);
            for (int q = 0; q < TPB / 32; ++q) tot = cadd<R>(tot, redsh[q]);
            part[(long long)s * gridDim.x + blockIdx.x] = cvt_to_d<R>(tot);
        }
    }
}

template <class R, int S>
__global__ void __launch_bounds__(TPB) k_matvec2(DevModel md, const int* __restrict__ sys_e, Sel sel, int nlist,
                                                const cx<R>* __restrict__ diag, const cx<R>* __restrict__ x, long long xs,
                                                cx<R>* __restrict__ y, long long ys, const double2* __restrict__ b,
                                                double2* __restrict__ part, int red) {
    __shared__ int offs[MV_MAXPTS];
    __shared__ cx<R> redsh[TPB / 32][S];
    const int nchunk = (md.Nnu + TPB - 1) / TPB;
    const int d = blockIdx.x / nchunk;
    const int nu = (blockIdx.x - d * nchunk) * TPB + threadIdx.x;
    const int N = md.N, Nnu = md.Nnu;
    const int pb = md.ebeg[d], np = min(md.ebeg[d + 1] - pb, MV_MAXPTS);
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const DevEntry& e = md.ent[pb + k];
        offs[k] = (e.dp - d) * Nnu + e.lin;
    }
    const cx<R>* xp[S];
    int sy[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const int li = blockIdx.y * S + k;
        int s = -1;
        if (li < nlist) {
            s = sel.list ? sel.list[li] : li;
            if (s >= 0 && sel.act && !sel.act[s]) s = -1;
        }
        sy[k] = s;
        xp[k] = x + (long long)(s < 0 ? 0 : s) * xs;
    }
    __syncthreads();
    const bool inr = nu < Nnu;
    const int i = d * Nnu + nu;
    cx<R> acc[S], xi[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
        acc[k] = mkc<R>(0, 0);
        xi[k] = mkc<R>(0, 0);
        if (sy[k] >= 0 && inr) {
            xi[k] = xp[k][i];
            acc[k] = cmul<R>(diag[(long long)sys_e[sy[k]] * N + i], xi[k]);
        }
    }
    if (inr) {
        const R* pc = pcp<R>(md) + (long long)pb * Nnu + nu;
        for (int k = 0; k < np; ++k) {
            const R c = __ldg(pc + (long long)k * Nnu);
            if (c != (R)0) {
                const int j = min(max(i + offs[k], 0), N - 1);
#pragma unroll
                for (int t = 0; t < S; ++t)
                    if (sy[t] >= 0) {
                        const cx<R> v = xp[t][j];
                        acc[t].x = fma(-c, v.x, acc[t].x);
                        acc[t].y = fma(-c, v.y, acc[t].y);
                    }
            }
        }
    }
    cx<R> loc[S];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        loc[t] = mkc<R>(0, 0);
        if (sy[t] >= 0 && inr) {
            cx<R> out = acc[t];
            if (b) {
                const double2 bb = b[(long long)sy[t] * N + i];
                out = mkc<R>((R)bb.x - out.x, (R)bb.y - out.y);
            }
            y[(long long)sy[t] * ys + i] = out;
            if (red == 1) loc[t] = cmul<R>(xi[t], out);
            else if (red == 2) {
                const float ox = (float)out.x, oy = (float)out.y;  // norm for the stopping test: FP32 suffices
                loc[t] = mkc<R>((R)(ox * ox + oy * oy), 0);
            }
        }
    }
    if (red) {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const cx<R> v = warp_sum_c<R>(loc[t]);
            if (lane == 0) redsh[w][t] = v;
        }
        __syncthreads();
        if (threadIdx.x < S && sy[threadIdx.x] >= 0) {
            cx<R> tot = mkc<R>(0, 0);
            for (int q = 0; q < TPB / 32; ++q) tot = cadd<R>(tot, redsh[q][threadIdx.x]);
            part[(long long)sy[threadIdx.x] * gridDim.x + blockIdx.x] = cvt_to_d<R>(tot);
        }
    }
}



// Register-blocked batched matvec: one thread owns EPT consecutive elements of one state and S
// systems.  For every stencil point it loads the EPT coefficients once and the EPT neighbours of
// each system from one base address, so the instruction count per element-system is a few per
// point; neighbour indices are clamped only for groups at the ends of the vector (their
// coefficients are zero there).  Same contract as k_matvec2; grid x = (state d, chunk of TPB*EPT
// elements), y = groups of S systems.
template <class R, int S, int EPT>
__global__ void __launch_bounds__(TPB) k_matvec3(DevModel md, const int* __restrict__ sys_e, Sel sel, int nlist,
                                                const cx<R>* __restrict__ diag, const cx<R>* __restrict__ x, long long xs,
                                                cx<R>* __restrict__ y, long long ys, const double2* __restrict__ b,
                                                double2* __restrict__ part, int red) {
    __shared__ int offs[MV_MAXPTS];
    __shared__ cx<R> redsh[TPB / 32][S];
    constexpr int T = TPB * EPT;
    const int Nnu = md.Nnu, N = md.N;
    const int nchunk = (Nnu + T - 1) / T;
    const int d = blockIdx.x / nchunk;
    const int nu0 = (blockIdx.x - d * nchunk) * T + threadIdx.x * EPT;
    const int pb = md.ebeg[d], np = min(md.ebeg[d + 1] - pb, MV_MAXPTS);
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const DevEntry& e = md.ent[pb + k];
        offs[k] = (e.dp - d) * Nnu + e.lin;
    }
    const cx<R>* xp[S];
    int sy[S];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const int li = blockIdx.y * S + t;
        int s = -1;
        if (li < nlist) {
            s = sel.list ? sel.list[li] : li;
            if (s >= 0 && sel.act && !sel.act[s]) s = -1;
        }
        sy[t] = s;
        xp[t] = x + (long long)(s < 0 ? 0 : s) * xs;
    }
    __syncthreads();
    const int nv = min(EPT, Nnu - nu0);  // elements of this thread inside the plane
    const int i0 = d * Nnu + nu0;
    cx<R> acc[S][EPT], xi[S][EPT];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const cx<R>* dg = diag + (long long)sys_e[sy[t] < 0 ? 0 : sy[t]] * N;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            xi[t][e] = mkc<R>(0, 0);
            acc[t][e] = mkc<R>(0, 0);
            if (sy[t] >= 0 && e < nv) {
                xi[t][e] = xp[t][i0 + e];
                acc[t][e] = cmul<R>(dg[i0 + e], xi[t][e]);
            }
        }
    }
    if (nv > 0) {
        const R* pc = pcp<R>(md) + (long long)pb * Nnu + nu0;
        for (int k = 0; k < np; ++k) {
            R c[EPT];
#pragma unroll
            for (int e = 0; e < EPT; ++e) c[e] = e < nv ? __ldg(pc + (long long)k * Nnu + e) : (R)0;
            const int j0 = i0 + offs[k];
            if (j0 >= 0 && j0 + EPT <= N) {
#pragma unroll
                for (int t = 0; t < S; ++t) {
                    const cx<R>* xb = xp[t] + j0;
#pragma unroll
                    for (int e = 0; e < EPT; ++e) {
                        const cx<R> v = xb[e];
                        acc[t][e].x = fma(-c[e], v.x, acc[t][e].x);
                        acc[t][e].y = fma(-c[e], v.y, acc[t][e].y);
                    }
                }
            } else {
#pragma unroll
                for (int t = 0; t < S; ++t) {
#pragma unroll
                    for (int e = 0; e < EPT; ++e) {
                        const cx<R> v = xp[t][min(max(j0 + e, 0), N - 1)];
                        acc[t][e].x = fma(-c[e], v.x, acc[t][e].x);
                        acc[t][e].y = fma(-c[e], v.y, acc[t][e].y);
                    }
                }
            }
        }
    }
    cx<R> loc[S];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        loc[t] = mkc<R>(0, 0);
        if (sy[t] < 0) continue;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            if (e >= nv) continue;
            cx<R> out = acc[t][e];
            if (b) {
                const double2 bb = b[(long long)sy[t] * N + i0 + e];
                out = mkc<R>((R)bb.x - out.x, (R)bb.y - out.y);
            }
            y[(long long)sy[t] * ys + i0 + e] = out;
            if (red == 1) loc[t] = cfma<R>(xi[t][e], out, loc[t]);
            else if (red == 2) {
                const float ox = (float)out.x, oy = (float)out.y;  // norm for the stopping test: FP32 suffices
                loc[t].x += (R)(ox * ox + oy * oy);
            }
        }
    }
    if (red) {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const cx<R> v = warp_sum_c<R>(loc[t]);
            if (lane == 0) redsh[w][t] = v;
        }
        __syncthreads();
        if (threadIdx.x < S && sy[threadIdx.x] >= 0) {
            cx<R> tot = mkc<R>(0, 0);
            for (int q = 0; q < TPB / 32; ++q) tot = cadd<R>(tot, redsh[q][threadIdx.x]);
            part[(long long)sy[threadIdx.x] * gridDim.x + blockIdx.x] = cvt_to_d<R>(tot);
        }
    }
}

// Windowed variant: the CTA stages, for each of its S systems and each state plane, the window
// of x its TPB*EPT elements reach (contiguous, [nu0 + lmin, nu0 + T + lmax)) in shared memory,
// together with the per-mode oscillator tables, so every neighbour and every coefficient factor
// is read from shared memory; global traffic is the window (about (1 + (lmax-lmin)/T) x), the
// diagonal table and y.  Coefficients are formed on the fly as coef * prod_m tab_m[n_m]; a
// neighbour outside the basis has a zero factor, and its window slot holds a finite value.
// Same contract as k_matvec2.
constexpr int MV_TAB_SMEM = 8192;  // most oscillator-table entries staged in shared memory

template <class R, int S, int EPT, int M>
__global__ void __launch_bounds__(TPB) k_matvec_tiled(DevModel md, int W_alloc, const int* __restrict__ sys_e, Sel sel,
                                                     int nlist, const cx<R>* __restrict__ diag, const cx<R>* __restrict__ x,
                                                     long long xs, cx<R>* __restrict__ y, long long ys,
                                                     const double2* __restrict__ b, double2* __restrict__ part, int red) {
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R>* win = reinterpret_cast<cx<R>*>(smraw);
    __shared__ R pcoef[MV_MAXPTS];
    __shared__ int plin[MV_MAXPTS];
    __shared__ int pdp[MV_MAXPTS];
    __shared__ short pcol[MV_MAXPTS][M];
    __shared__ cx<R> redsh[TPB / 32][S];
    constexpr int T = TPB * EPT;
    const int Nnu = md.Nnu, N = md.N, ns = md.ns;
    const int nchunk = (Nnu + T - 1) / T;
    const int d = blockIdx.x / nchunk;
    const int nu0 = (blockIdx.x - d * nchunk) * T;
    const int lmin = md.lmin[d], W = W_alloc, base = nu0 + lmin;
    const int pb = md.ebeg[d], np = min(md.ebeg[d + 1] - pb, MV_MAXPTS);
    // dynamic shared memory: S * ns windows of W entries, then the oscillator tables
    R* stab = reinterpret_cast<R*>(win + (long long)S * ns * W_alloc);
    const R* gtab = tabp<R>(md);
    for (int k = threadIdx.x; k < md.ntab; k += blockDim.x) stab[k] = gtab[k];
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const DevEntry& e = md.ent[pb + k];
        plin[k] = e.lin;  // window position of the neighbour: (nu + lin) - base = rel + lin
        pdp[k] = e.dp;
        pcoef[k] = (R)e.coef;
#pragma unroll
        for (int m = 0; m < M; ++m) pcol[k][m] = (short)e.col[m];
    }
    int sy[S];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const int li = blockIdx.y * S + t;
        int s = -1;
        if (li < nlist) {
            s = sel.list ? sel.list[li] : li;
            if (s >= 0 && sel.act && !sel.act[s]) s = -1;
        }
        sy[t] = s;
    }
    // stage the windows
#pragma unroll
    for (int t = 0; t < S; ++t) {
        if (sy[t] < 0) continue;
        for (int dp = 0; dp < ns; ++dp) {
            cx<R>* w = win + (long long)(t * ns + dp) * W;
            const cx<R>* src = x + (long long)sy[t] * xs + (long long)dp * Nnu;
            for (int q = threadIdx.x; q < W; q += TPB) {
                const int g = base + q;
                w[q] = (g >= 0 && g < Nnu) ? src[g] : mkc<R>(0, 0);
            }
        }
    }
    __syncthreads();
    cx<R> loc[S];
#pragma unroll
    for (int t = 0; t < S; ++t) loc[t] = mkc<R>(0, 0);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int nu = nu0 + threadIdx.x + e * TPB;
        if (nu >= Nnu) break;
        const int i = d * Nnu + nu;
        const int rel = nu - base;
        int n[MAXM];
        decode<M>(md, nu, n);
        cx<R> acc[S], xi[S];
#pragma unroll
        for (int t = 0; t < S; ++t) {
            xi[t] = mkc<R>(0, 0);
            acc[t] = mkc<R>(0, 0);
            if (sy[t] >= 0) {
                xi[t] = win[(long long)(t * ns + d) * W + rel];
                acc[t] = cmul<R>(diag[(long long)sys_e[sy[t]] * N + i], xi[t]);
            }
        }
        for (int k = 0; k < np; ++k) {
            R c = pcoef[k];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int col = pcol[k][m];
                if (col >= 0) c *= stab[col + n[m]];
            }
            const int widx = pdp[k] * W + rel + plin[k];
#pragma unroll
            for (int t = 0; t < S; ++t) {
                const cx<R> v = win[(long long)t * ns * W + widx];
                acc[t].x = fma(-c, v.x, acc[t].x);
                acc[t].y = fma(-c, v.y, acc[t].y);
            }
        }
#pragma unroll
        for (int t = 0; t < S; ++t) {
            if (sy[t] < 0) continue;
            cx<R> out = acc[t];
            if (b) {
                const double2 bb = b[(long long)sy[t] * N + i];
                out = mkc<R>((R)bb.x - out.x, (R)bb.y - out.y);
            }
            y[(long long)sy[t] * ys + i] = out;
            if (red == 1) loc[t] = cfma<R>(xi[t], out, loc[t]);
            else if (red == 2) {
                const float ox = (float)out.x, oy = (float)out.y;  // norm for the stopping test: FP32 suffices
                loc[t].x += (R)(ox * ox + oy * oy);
            }
        }
    }
    if (red) {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const cx<R> v = warp_sum_c<R>(loc[t]);
            if (lane == 0) redsh[w][t] = v;
        }
        __syncthreads();
        if (threadIdx.x < S && sy[threadIdx.x] >= 0) {
            cx<R> tot = mkc<R>(0, 0);
            for (int q = 0; q < TPB / 32; ++q) tot = cadd<R>(tot, redsh[q][threadIdx.x]);
            part[(long long)sy[threadIdx.x] * gridDim.x + blockIdx.x] = cvt_to_d<R>(tot);
        }
    }
}

// Windowed batched matvec with every state of a tile in one CTA.  A CTA owns T = TPB * EPT
// consecutive vibrational indices nu of all n_s states for S systems: it stages, per system and
// state, the window [nu0 + lo, nu0 + T + hi) of x that the stencil reaches (lo, hi: smallest and
// largest in-plane offset of any point) into shared memory with cp.async (zero-filled outside
// the basis), so every entry of x leaves L2/HBM about (T + hi - lo) / T times and every staged
// window serves all the states that read it.  Coefficients come from the primary-mode rows of
// the stencil (rct: -coef (q^k)_{n, n + delta}, energy-independent) held in shared memory, times
// the oscillator table of a secondary mode where a point has one; nothing is streamed per system
// but x, y and the diagonal table (read once for the systems of the CTA that share an energy).
// Same contract as k_matvec2 (y = A x or b - A x, optional partials per system and CTA).
template <class R> __device__ __forceinline__ const R* wrows(const DevModel& md);
template <> __device__ __forceinline__ const float* wrows<float>(const DevModel& md) {
    return reinterpret_cast<const float*>(md.rct);  // packed pairs (-c, -c)
}
template <> __device__ __forceinline__ const double* wrows<double>(const DevModel& md) { return md.rct64; }

template <class R> __device__ __forceinline__ void cp_async_cx(unsigned dst, const void* src, bool ok) {
    const int n = ok ? (int)sizeof(cx<R>) : 0;  // 0 source bytes: the destination is zero-filled
    if constexpr (sizeof(cx<R>) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

// acc += c * v for a real coefficient c (float: the packed pair (c, c) from the row)
__device__ __forceinline__ float2 wfma(float2 c, float2 v, float2 acc) { return ffma2(c, v, acc); }
__device__ __forceinline__ double2 wfma(double c, double2 v, double2 acc) {
    return make_double2(fma(c, v.x, acc.x), fma(c, v.y, acc.y));
}

template <class R, int S, int EPT, int M>
__global__ void __launch_bounds__(TPB) k_matvec_win(DevModel md, int lo, int Wst, const int* __restrict__ sys_e, Sel sel,
                                                   int nlist, const cx<R>* __restrict__ diag, const cx<R>* __restrict__ x,
                                                   long long xs, cx<R>* __restrict__ y, long long ys,
                                                   const double2* __restrict__ b, double2* __restrict__ part, int red) {
    using C = cx<R>;
    using CR = typename std::conditional<sizeof(R) == 4, float2, double>::type;  // row entry type
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ C redsh[TPB / 32][S];
    constexpr int T = TPB * EPT;
    const int Nnu = md.Nnu, N = md.N, ns = md.ns, tid = threadIdx.x;
    const int nu0 = blockIdx.x * T, base = nu0 + lo;
    const size_t wbytes = (((size_t)S * ns * Wst * sizeof(C)) + 15) & ~size_t(15);
    const size_t rbytes = (((size_t)md.nrct * 8) + 15) & ~size_t(15);
    const CR* rows = reinterpret_cast<const CR*>(smraw + wbytes);
    int4* sdesc = reinterpret_cast<int4*>(smraw + wbytes + rbytes);
    int sy[S], se[S];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const int li = blockIdx.y * S + t;
        int s = -1;
        if (li < nlist) {
            s = sel.list ? sel.list[li] : li;
            if (s >= 0 && sel.act && !sel.act[s]) s = -1;
        }
        sy[t] = s;
        se[t] = s < 0 ? -1 : sys_e[s];
    }
    // stage the windows (asynchronous copies), the coefficient rows and the point descriptors
    const unsigned wsh = (unsigned)__cvta_generic_to_shared(smraw);
#pragma unroll
    for (int t = 0; t < S; ++t)
        for (int dp = 0; dp < ns; ++dp) {
            const C* src = x + (long long)(sy[t] < 0 ? 0 : sy[t]) * xs + (long long)dp * Nnu;
            const unsigned dst = wsh + (unsigned)(((t * ns + dp) * Wst) * sizeof(C));
            for (int q = tid; q < Wst; q += TPB) {
                const int g = base + q;
                const bool ok = sy[t] >= 0 && g >= 0 && g < Nnu;
                cp_async_cx<R>(dst + (unsigned)(q * sizeof(C)), ok ? (const void*)(src + g) : (const void*)x, ok);
            }
        }
    asm volatile("cp.async.commit_group;" ::: "memory");
    {
        const CR* grow = reinterpret_cast<const CR*>(wrows<R>(md));
        CR* srow = const_cast<CR*>(rows);
        for (int k = tid; k < md.nrct; k += TPB) srow[k] = grow[k];
        for (int k = tid; k < md.rbeg[ns]; k += TPB) {
            const int4 w = md.wdesc[k];
            sdesc[k] = make_int4(w.x, (int)sizeof(C) * ((w.w >> 8) * Wst + w.y), w.z, w.w & 0xff);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const R* tab = tabp<R>(md);
    const unsigned char* win = smraw;
    const size_t tstride = (size_t)ns * Wst * sizeof(C);  // bytes between the windows of two systems
    C loc[S];
#pragma unroll
    for (int t = 0; t < S; ++t) loc[t] = mkc<R>(0, 0);
    for (int d = 0; d < ns; ++d) {
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int nu = nu0 + e * TPB + tid;
            if (nu >= Nnu) break;
            const int i = d * Nnu + nu;
            int n[MAXM];
            decode<M>(md, nu, n);
            // window slot of nu in the state-0 window of system 0; state dp's slot lies dp * Wst
            // entries further (the descriptors' byte offsets q.y include dp * Wst + lin)
            const unsigned char* wc = win + (size_t)(nu - base) * sizeof(C);
            const size_t dself = (size_t)d * Wst * sizeof(C);
            C acc[S], xi[S];
            const C dg0 = se[0] >= 0 ? diag[(long long)se[0] * N + i] : mkc<R>(0, 0);
#pragma unroll
            for (int t = 0; t < S; ++t) {
                xi[t] = *reinterpret_cast<const C*>(wc + t * tstride + dself);
                const C dg = (t == 0 || se[t] == se[0]) ? dg0 : diag[(long long)(se[t] < 0 ? 0 : se[t]) * N + i];
                acc[t] = cmul<R>(dg, xi[t]);
            }
            int k = md.rbeg[d];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int kend = k + md.rcnt[d][m];
                const unsigned char* row = reinterpret_cast<const unsigned char*>(rows) + (size_t)n[m] * 8;
#pragma unroll 4
                for (; k < kend; ++k) {
                    const int4 q = sdesc[k];
                    CR c = *reinterpret_cast<const CR*>(row + q.x);
                    if (q.z >= 0) {  // a second mode's factor (bilinear terms)
                        const R f = tab[q.z + nsel<M>(n, q.w)];
                        if constexpr (sizeof(R) == 4) c = make_float2(c.x * f, c.y * f);
                        else c *= f;
                    }
#pragma unroll
                    for (int t = 0; t < S; ++t)  // neighbours outside the basis read zero-filled slots
                        acc[t] = wfma(c, *reinterpret_cast<const C*>(wc + t * tstride + q.y), acc[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < S; ++t) {
                if (sy[t] < 0) continue;
                C out = acc[t];
                if (b) {
                    const double2 bb = b[(long long)sy[t] * N + i];
                    out = mkc<R>((R)bb.x - out.x, (R)bb.y - out.y);
                }
                y[(long long)sy[t] * ys + i] = out;
                if (red == 1) loc[t] = cfma<R>(xi[t], out, loc[t]);
                else if (red == 2) {
                    const float ox = (float)out.x, oy = (float)out.y;  // norm for the stopping test: FP32 suffices
                    loc[t].x += (R)(ox * ox + oy * oy);
                }
            }
        }
    }
    if (red) {
        const int lane = tid & 31, w = tid >> 5;
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const C v = warp_sum_c<R>(loc[t]);
            if (lane == 0) redsh[w][t] = v;
        }
        __syncthreads();
        if (tid < S && sy[tid] >= 0) {
            C tot = mkc<R>(0, 0);
            for (int q = 0; q < TPB / 32; ++q) tot = cadd<R>(tot, redsh[q][tid]);
            part[(long long)sy[tid] * gridDim.x + blockIdx.x] = cvt_to_d<R>(tot);
        }
    }
}


// ---------------------------------------------------------------- block preconditioner
struct PlanDev {
    int L, nblk, p, span;
    const int* chain_off;   // [L]   element offset of chain position c (relative)
    const int* fixed_base;  // [nblk] element index of chain position 0 of each block
    const int* ent_dc;      // [n off-diagonal points] chain offset of the point, 0 if outside
    // staging through shared memory (blocks whose chain contains the fastest mode): the chain
    // of a block is `nrun` contiguous runs of `runlen` elements; element k of run r sits at
    // base + run_off[r] + k and has chain position run_c0[r] + k * cs_run.
    int nrun, runlen, cs_run;
    const int* run_off;
    const int* run_c0;
    // wide bands (p > PMAX): level size and level count of the block-pentadiagonal form
    int S, K;
    // sandwich entries inside a block (q-dependent couplings): 5 ints each (see BlockPlan::sw_combo)
    const int* swc;
    int nswc;
};

// Entries of the sandwich operator in row (d, nu) of a block (Eq. FE): for every combination of
// a point k of P_j and a point k2 of P_j', the value spc[k][nu] g_(j,j')(nu + lin_k) spc[k2][nu + lin_k]
// at chain offset dc; `add(dc, v)` receives -v (A = ... - F).  Zero coefficients mark neighbours
// outside the basis.
template <class R, class Add>
__device__ __forceinline__ void sand_block_row(const DevModel& md, const PlanDev& pl, int e, int d, int nu, Add add) {
    const R* sp = spcp<R>(md);
    for (int t = 0; t < pl.nswc; ++t) {
        const int* cb = pl.swc + 5 * t;
        if (cb[0] != d) continue;
        const int k = cb[1], k2 = cb[2];
        const R c1 = sp[(long long)k * md.Nnu + nu];
        if (c1 == (R)0) continue;
        const int kap = nu + md.sp_lin[k];
        const R c2 = sp[(long long)k2 * md.Nnu + kap];
        if (c2 == (R)0) continue;
        const cx<R> g = sgp<R>(md)[((long long)e * md.npair + cb[3]) * md.Nnu + kap];
        add(cb[4], mkc<R>(-c1 * c2 * g.x, -c1 * c2 * g.y));
    }
}

// B = L D L^T of every block of every energy (Sec. III.B: factors computed once and stored).
// One thread per (energy, block); F[e][c][k][blk]: k = 0 holds 1/D_c, k >= 1 holds L_{c,c-k}.
template <class R, int M>
__global__ void k_block_factor(DevModel md, PlanDev pl, int nE, const cx<R>* __restrict__ diag, cx<R>* __restrict__ F,
                               int* __restrict__ fail) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nE * pl.nblk) return;
    const int e = (int)(t / pl.nblk), blk = (int)(t - (long long)e * pl.nblk);
    const int L = pl.L, p = pl.p, nblk = pl.nblk;
    const int base = pl.fixed_base[blk];
    const R* tab = tabp<R>(md);
    cx<R>* Fe = F + (long long)e * L * (p + 1) * nblk;
    auto Fat = [&](int c, int k) -> cx<R>& { return Fe[((long long)c * (p + 1) + k) * nblk + blk]; };
    cx<R> Dw[PMAX + 1];  // D of the last p rows (rolling)
    cx<R> row[PMAX + 1];
    bool bad = false;
    for (int c = 0; c < L; ++c) {
        const int i = base + pl.chain_off[c];
        const int d = i / md.Nnu, nu = i - d * md.Nnu;
        int n[MAXM];
        decode<M>(md, nu, n);
        for (int k = 0; k <= p; ++k) row[k] = mkc<R>(0, 0);
        row[0] = diag[(long long)e * md.N + i];
        for (int k = md.ebeg[d]; k < md.ebeg[d + 1]; ++k) {
            const int dc = pl.ent_dc[k];
            if (dc >= 0 || dc < -p || c + dc < 0) continue;
            const DevEntry pt = md.ent[k];
            R cf;
            if (point_coef<R, M>(pt, n, md, tab, cf)) row[-dc].x -= cf;
        }
        if (pl.nswc)
            sand_block_row<R>(md, pl, e, d, nu, [&](int dc, cx<R> v) {
                if (dc < 0 && dc >= -p && c + dc >= 0) row[-dc] = cadd<R>(row[-dc], v);
            });
        // row[k] now holds B[c][c-k]; eliminate left to right
        for (int jj = max(0, c - p); jj < c; ++jj) {
            const int kj = c - jj;
            cx<R> sacc = row[kj];
            for (int tt = max(max(0, c - p), jj - p); tt < jj; ++tt) {
                const cx<R> lct = row[c - tt];           // L[c][tt] (final)
                const cx<R> ljt = Fat(jj, jj - tt);       // L[jj][tt]
                sacc = csub<R>(sacc, cmul<R>(cmul<R>(lct, Dw[tt % (PMAX + 1)]), ljt));
            }
            row[kj] = cmul<R>(sacc, Fat(jj, 0));          // / D[jj]
        }
        cx<R> dc0 = row[0];
        for (int tt = max(0, c - p); tt < c; ++tt) {
            const cx<R> l = row[c - tt];
            dc0 = csub<R>(dc0, cmul<R>(cmul<R>(l, l), Dw[tt % (PMAX + 1)]));
        }
        cx<R> inv;
        const R a2 = cabs2<R>(dc0);
        if (!(a2 > (R)0) || !isfinite(a2)) {
            bad = true;
            inv = mkc<R>(0, 0);
        } else {
            inv = mkc<R>(dc0.x / a2, -dc0.y / a2);
        }
        Dw[c % (PMAX + 1)] = dc0;
        Fat(c, 0) = inv;
        for (int k = 1; k <= p; ++k) Fat(c, k) = (k <= c) ? row[k] : mkc<R>(0, 0);
    }
    if (bad) atomicExch(fail + e, 1);
}

// z = B^-1 r for every block of every active system; optional fused rz = r^T z partials.
// Grid: (ceil(nblk / BTPB), nsys).
template <class R>
__global__ void __launch_bounds__(BTPB) k_block_apply(PlanDev pl, const int* __restrict__ sys_e, Sel sel,
                                                     const cx<R>* __restrict__ F, const cx<R>* __restrict__ r, long long rs,
                                                     cx<R>* __restrict__ z, long long zs, double2* __restrict__ part) {
    __shared__ cx<R> sh[32];
    const int s = sel_sys(sel);
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    const int L = pl.L, p = pl.p, nblk = pl.nblk;
    cx<R> loc = mkc<R>(0, 0);
    if (blk < nblk) {
        const int e = sys_e[s];
        const cx<R>* Fe = F + (long long)e * L * (p + 1) * nblk + blk;
        const cx<R>* rv = r + (long long)s * rs;
        cx<R>* zv = z + (long long)s * zs;
        const int base = pl.fixed_base[blk];
        // forward: w_c = r_c - sum_k L[c][c-k] w_{c-k}
        for (int c = 0; c < L; ++c) {
            cx<R> w = rv[base + pl.chain_off[c]];
            const int kmax = min(p, c);
            for (int k = 1; k <= kmax; ++k)
                w = csub<R>(w, cmul<R>(Fe[((long long)c * (p + 1) + k) * nblk], zv[base + pl.chain_off[c - k]]));
            zv[base + pl.chain_off[c]] = w;
        }
        // backward: z_c = w_c / D_c - sum_k L[c+k][c] z_{c+k}
        for (int c = L - 1; c >= 0; --c) {
            const int ic = base + pl.chain_off[c];
            cx<R> v = cmul<R>(zv[ic], Fe[((long long)c * (p + 1)) * nblk]);
            const int kmax = min(p, L - 1 - c);
            for (int k = 1; k <= kmax; ++k)
                v = csub<R>(v, cmul<R>(Fe[((long long)(c + k) * (p + 1) + k) * nblk], zv[base + pl.chain_off[c + k]]));
            zv[ic] = v;
            if (part) {
                loc = cfma<R>(rv[ic], v, loc);
            }
        }
    }
    if (part) {
        const double2 tot = block_sum_c<R>(loc, sh);
        if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = tot;
    }
}


// ------------------------------------------------------------- staged block preconditioner
// z = B^-1 r for G consecutive blocks of one system per CTA.  The chains are gathered into
// shared memory with coalesced loads over their contiguous runs (tile[c][b], b fastest,
// padded), walked by one thread per block with a register window of P (>= p) previous
// values, and scattered back.  With `upd`, the COCG update x += alpha p, r -= alpha q is
// applied to the gathered elements first (partials ||r||^2).  r^T z = sum_c w_c^2 / D_c
// with w = L^-1 r is accumulated in the forward sweep (partials part_rz).
constexpr int SG = 32;       // blocks (chains) per CTA
constexpr int STPB = 128;    // threads per CTA

template <class R, int P>
__global__ void __launch_bounds__(STPB) k_block_staged(PlanDev pl, const int* __restrict__ alist, const int* __restrict__ act,
                                                      const int* __restrict__ sys_e, const cx<R>* __restrict__ F,
                                                      const SysState* __restrict__ st, int upd, cx<R>* __restrict__ x,
                                                      cx<R>* __restrict__ r, long long rs, const cx<R>* __restrict__ pv,
                                                      const cx<R>* __restrict__ q, cx<R>* __restrict__ z, long long zs,
                                                      double2* __restrict__ part_rr, double2* __restrict__ part_rz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
    __shared__ cx<R> sh[32];
    const int s = alist ? alist[blockIdx.y] : blockIdx.y;
    if (s < 0 || (act && !act[s])) return;
    const int L = pl.L, p = pl.p, nblk = pl.nblk;
    const int b0 = blockIdx.x * SG;
    const int G = min(SG, nblk - b0);
    const int e = sys_e[s];
    const int runlen = pl.runlen, nrun = pl.nrun, csr = pl.cs_run;
    cx<R>* rv = r + (long long)s * rs;
    cx<R>* zv = z + (long long)s * zs;
    const long long so = (long long)s * (long long)(upd ? rs : 0);
    cx<R> al = mkc<R>(0, 0);
    if (upd) al = cvt_from_d<R>(st[s].alpha);
    // ---- gather (and update)
    R lrr = 0;
    const int tot = G * nrun * runlen;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int k = idx % runlen;
        const int t2 = idx / runlen;
        const int rr_ = t2 % nrun, b = t2 / nrun;
        const long long el = (long long)pl.fixed_base[b0 + b] + pl.run_off[rr_] + k;
        cx<R> rvv = rv[el];
        if (upd) {
            const cx<R> xv = x[so + el], pp = pv[so + el], qq = q[so + el];
            x[so + el] = cfma<R>(al, pp, xv);
            rvv = csub<R>(rvv, cmul<R>(al, qq));
            rv[el] = rvv;
            lrr += cabs2<R>(rvv);
        }
        tile[(pl.run_c0[rr_] + k * csr) * (SG + 1) + b] = rvv;
    }
    __syncthreads();
    // ---- chain walk: thread b < G owns block b0 + b
    cx<R> lrz = mkc<R>(0, 0);
    if (threadIdx.x < G) {
        const int b = threadIdx.x;
        const cx<R>* Fe = F + (long long)e * L * (p + 1) * nblk + b0 + b;
        cx<R> win[P];
#pragma unroll
        for (int k = 0; k < P; ++k) win[k] = mkc<R>(0, 0);
        cx<R> Lr[P + 1], Ln[P + 1];
#pragma unroll
        for (int k = 0; k <= P; ++k) Lr[k] = (k <= p) ? Fe[(long long)k * nblk] : mkc<R>(0, 0);
        for (int c = 0; c < L; ++c) {
            // prefetch the next factor row
#pragma unroll
            for (int k = 0; k <= P; ++k)
                Ln[k] = (k <= p && c + 1 < L) ? Fe[((long long)(c + 1) * (p + 1) + k) * nblk] : mkc<R>(0, 0);
            cx<R> w = tile[c * (SG + 1) + b];
#pragma unroll
            for (int k = P; k >= 1; --k) w = csub<R>(w, cmul<R>(Lr[k], win[k - 1]));
            const cx<R> v = cmul<R>(w, Lr[0]);
            lrz = cfma<R>(w, v, lrz);
            tile[c * (SG + 1) + b] = v;
#pragma unroll
            for (int k = P - 1; k >= 1; --k) win[k] = win[k - 1];
            win[0] = w;
#pragma unroll
            for (int k = 0; k <= P; ++k) Lr[k] = Ln[k];
        }
        // backward: z_c = v_c - sum_k L[c+k][c] z_{c+k}
#pragma unroll
        for (int k = 0; k < P; ++k) win[k] = mkc<R>(0, 0);
        cx<R> Lc[P + 1], Lcn[P + 1];
#pragma unroll
        for (int k = 1; k <= P; ++k)
            Lc[k] = (k <= p && L - 1 + k < L) ? Fe[((long long)(L - 1 + k) * (p + 1) + k) * nblk] : mkc<R>(0, 0);
        for (int c = L - 1; c >= 0; --c) {
#pragma unroll
            for (int k = 1; k <= P; ++k)
                Lcn[k] = (k <= p && c >= 1 && c - 1 + k < L) ? Fe[((long long)(c - 1 + k) * (p + 1) + k) * nblk] : mkc<R>(0, 0);
            cx<R> zz = tile[c * (SG + 1) + b];
#pragma unroll
            for (int k = P; k >= 1; --k) zz = csub<R>(zz, cmul<R>(Lc[k], win[k - 1]));
            tile[c * (SG + 1) + b] = zz;
#pragma unroll
            for (int k = P - 1; k >= 1; --k) win[k] = win[k - 1];
            win[0] = zz;
#pragma unroll
            for (int k = 1; k <= P; ++k) Lc[k] = Lcn[k];
        }
    }
    __syncthreads();
    // ---- scatter
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int k = idx % runlen;
        const int t2 = idx / runlen;
        const int rr_ = t2 % nrun, b = t2 / nrun;
        const long long el = (long long)pl.fixed_base[b0 + b] + pl.run_off[rr_] + k;
        zv[el] = tile[(pl.run_c0[rr_] + k * csr) * (SG + 1) + b];
    }
    if (part_rr) {
        const double2 t = block_sum_c<R>(mkc<R>(lrr, 0), sh);
        if (threadIdx.x == 0) part_rr[(long long)s * gridDim.x + blockIdx.x] = t;
    }
    if (part_rz) {
        const double2 t = block_sum_c<R>(lrz, sh);
        if (threadIdx.x == 0) part_rz[(long long)s * gridDim.x + blockIdx.x] = t;
    }
}

// --------------------------------------------------------- wide-band block preconditioner
// Blocks whose chain half bandwidth p exceeds PMAX (the states x two-dimensional bend blocks of
// a CO2-type model: 3 * 20 * 20 = 1200 unknowns with p = 120) are factored in LEVELS of S
// consecutive chain positions, S = 4 ceil(p / 8) >= p / 2, so that B is block pentadiagonal
// with S x S blocks: B = L D L^T with L unit block-lower (blocks L_{k+1,k}, L_{k+2,k}) and D
// block diagonal (dense complex symmetric S x S).  The last level is padded with identity
// rows.  Per energy and block the factor holds, for every level k, five S x S blocks:
//   [0] D_k^-1 (symmetrized), [1], [2] Lf_j = L_{k,k-j}^T, [3], [4] Lb_j = L_{k+j,k}
// (all row-major), so that thread i of a solve reads column i of each (coalesced).  Both
// triangular sweeps are then dense block products, K = ceil(L / S) sequential steps instead
// of L scalar ones.  After the factors, each energy holds a workspace of 9 S x S blocks per
// block (the Schur-complement window during the factorization).
constexpr int LF_THREADS = 256;  // threads of the level factorization
constexpr int LV_SMAX = 80;      // largest level (p <= 160 = PWMAX)
static_assert(4 * ((PWMAX + 7) / 8) <= LV_SMAX, "PWMAX needs a larger level size");

__host__ __device__ inline int level_size(int p) { return 4 * ((p + 7) / 8); }
__host__ __device__ inline long long level_factor_entries(int nblk, int K, int S) {
    return (long long)nblk * S * S * (5LL * K + 9);
}

// Rows of level a of B (chain positions a S .. a S + S - 1) into the window blocks W(a, a),
// W(a, a - 1), W(a, a - 2) (those with a - j >= 0): Wslot(a, b) = W + ((a % 3) * 3 + b % 3) S^2.
template <class R, int M>
__device__ void level_assemble(const DevModel& md, const PlanDev& pl, int e, int blk, int a, const cx<R>* __restrict__ diag,
                               cx<R>* __restrict__ W) {
    const int S = pl.S, L = pl.L;
    const long long S2 = (long long)S * S;
    for (int j = 0; j <= 2 && a - j >= 0; ++j) {
        cx<R>* Wb = W + ((a % 3) * 3 + (a - j) % 3) * S2;
        for (long long t = threadIdx.x; t < S2; t += blockDim.x) Wb[t] = mkc<R>(0, 0);
    }
    __syncthreads();
    const R* tab = tabp<R>(md);
    for (int r = threadIdx.x; r < S; r += blockDim.x) {
        const int c = a * S + r;
        cx<R>* Waa = W + ((a % 3) * 3 + a % 3) * S2;
        if (c >= L) {  // padding: identity
            Waa[(long long)r * S + r] = mkc<R>(1, 0);
            continue;
        }
        const int i = pl.fixed_base[blk] + pl.chain_off[c];
        const int d = i / md.Nnu, nu = i - d * md.Nnu;
        int n[MAXM];
        decode<M>(md, nu, n);
        Waa[(long long)r * S + r] = diag[(long long)e * md.N + i];
        for (int k = md.ebeg[d]; k < md.ebeg[d + 1]; ++k) {
            const int dc = pl.ent_dc[k];
            if (dc == 0) continue;
            const int cp = c + dc;
            if (cp < 0 || cp >= L) continue;
            const int b = cp / S;
            if (b < a - 2 || b > a) continue;
            R cf;
            if (point_coef<R, M>(md.ent[k], n, md, tab, cf)) {
                cx<R>& dst = W[((a % 3) * 3 + b % 3) * S2 + (long long)r * S + (cp - b * S)];
                dst.x -= cf;
            }
        }
        if (pl.nswc)
            sand_block_row<R>(md, pl, e, d, nu, [&](int dc, cx<R> v) {
                const int cp = c + dc;
                if (cp < 0 || cp >= L) return;
                const int b = cp / S;
                if (b < a - 2 || b > a) return;
                cx<R>& dst = W[((a % 3) * 3 + b % 3) * S2 + (long long)r * S + (cp - b * S)];
                dst = cadd<R>(dst, v);
            });
    }
}

// C = X Y for S x S matrices in shared memory (row-major), 2 x 2 output tiles per thread;
// `emit(r, c, v)` receives every entry of C.
template <class R, class Emit>
__device__ __forceinline__ void level_gemm(int S, const cx<R>* X, const cx<R>* Y, Emit emit) {
    const int nt = S / 2;
    for (int t = threadIdx.x; t < nt * nt; t += blockDim.x) {
        const int r0 = (t / nt) * 2, c0 = (t % nt) * 2;
        cx<R> a00 = mkc<R>(0, 0), a01 = a00, a10 = a00, a11 = a00;
        for (int m = 0; m < S; ++m) {
            const cx<R> x0 = X[r0 * S + m], x1 = X[(r0 + 1) * S + m];
            const cx<R> y0 = Y[m * S + c0], y1 = Y[m * S + c0 + 1];
            a00 = cfma<R>(x0, y0, a00);
            a01 = cfma<R>(x0, y1, a01);
            a10 = cfma<R>(x1, y0, a10);
            a11 = cfma<R>(x1, y1, a11);
        }
        emit(r0, c0, a00);
        emit(r0, c0 + 1, a01);
        emit(r0 + 1, c0, a10);
        emit(r0 + 1, c0 + 1, a11);
    }
}

// Block L D L^T of one preconditioner block per CTA (grid: blocks x energies), right-looking
// over levels (Sec. III.B: the factors are computed once per energy and stored):
//   D_k^-1 by Gauss-Jordan elimination with partial pivoting,
//   L_{k+j,k} = W(k+j, k) D_k^-1 (j = 1, 2),
//   W(k+i, k+j) -= L_{k+i,k} W(k+j, k)^T (1 <= j <= i <= 2),
// then the rows of level k + 3 enter the window.  A zero pivot sets fail[e].
template <class R, int M>
__global__ void __launch_bounds__(LF_THREADS) k_level_factor(DevModel md, PlanDev pl, const cx<R>* __restrict__ diag,
                                                            cx<R>* __restrict__ F, int* __restrict__ fail) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* sm = reinterpret_cast<cx<R>*>(smem_raw);  // 2 S^2 entries
    __shared__ int piv_sh, bad_sh;
    __shared__ cx<R> pinv_sh;
    const int S = pl.S, K = pl.K, blk = blockIdx.x, e = blockIdx.y;
    const long long S2 = (long long)S * S;
    cx<R>* Fe = F + (long long)e * level_factor_entries(pl.nblk, K, S);
    cx<R>* Out = Fe + (long long)blk * K * 5 * S2;
    cx<R>* W = Fe + (long long)pl.nblk * K * 5 * S2 + (long long)blk * 9 * S2;
    auto slot = [&](int a, int b) { return W + ((a % 3) * 3 + b % 3) * S2; };
    auto out = [&](int k, int part) { return Out + ((long long)k * 5 + part) * S2; };
    if (threadIdx.x == 0) bad_sh = 0;
    for (int a = 0; a < 3 && a < K; ++a) level_assemble<R, M>(md, pl, e, blk, a, diag, W);
    for (int k = 0; k < K; ++k) {
        __syncthreads();
        // ---- D_k^-1: [D | I] -> [I | D^-1] in shared memory (row stride 2 S)
        cx<R>* aug = sm;
        const cx<R>* D = slot(k, k);
        for (long long t = threadIdx.x; t < 2 * S2; t += blockDim.x) {
            const int r = (int)(t / (2 * S)), c = (int)(t - (long long)r * 2 * S);
            aug[t] = c < S ? D[(long long)r * S + c] : mkc<R>(c - S == r ? 1 : 0, 0);
        }
        __syncthreads();
        for (int m = 0; m < S; ++m) {
            if (threadIdx.x < 32) {
                R best = (R)-1;
                int bi = m;
                for (int r = m + threadIdx.x; r < S; r += 32) {
                    const R v = cabs2<R>(aug[(long long)r * 2 * S + m]);
                    if (v > best) {
                        best = v;
                        bi = r;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const R ob = __shfl_down_sync(0xffffffffu, best, o);
                    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                }
                if (threadIdx.x == 0) {
                    piv_sh = bi;
                    const cx<R> pv = aug[(long long)bi * 2 * S + m];
                    const R a2 = cabs2<R>(pv);
                    if (!(a2 > (R)0) || !isfinite(a2)) {
                        bad_sh = 1;
                        pinv_sh = mkc<R>(0, 0);
                    } else {
                        pinv_sh = mkc<R>(pv.x / a2, -pv.y / a2);
                    }
                }
            }
            __syncthreads();
            const int pr = piv_sh;
            const cx<R> pinv = pinv_sh;
            for (int c = threadIdx.x; c < 2 * S; c += blockDim.x) {
                const cx<R> vp = aug[(long long)pr * 2 * S + c];
                if (pr != m) aug[(long long)pr * 2 * S + c] = aug[(long long)m * 2 * S + c];
                aug[(long long)m * 2 * S + c] = cmul<R>(vp, pinv);
            }
            __syncthreads();
            const int w = 2 * S - m - 1;  // columns m + 1 .. 2 S - 1
            for (long long t = threadIdx.x; t < (long long)S * w; t += blockDim.x) {
                const int r = (int)(t / w), c = m + 1 + (int)(t - (long long)r * w);
                if (r == m) continue;
                const cx<R> f = aug[(long long)r * 2 * S + m];
                aug[(long long)r * 2 * S + c] = csub<R>(aug[(long long)r * 2 * S + c], cmul<R>(f, aug[(long long)m * 2 * S + c]));
            }
            __syncthreads();
        }
        // D_k^-1 is complex symmetric; its symmetric part is stored so that the preconditioner
        // L^-T D^-1 L^-1 stays exactly symmetric under rounding (COCG relies on it)
        cx<R>* Dt = out(k, 0);
        for (long long t = threadIdx.x; t < S2; t += blockDim.x) {
            const int r = (int)(t / S), c = (int)(t - (long long)r * S);
            const cx<R> a = aug[(long long)r * 2 * S + S + c], b = aug[(long long)c * 2 * S + S + r];
            Dt[t] = mkc<R>((R)0.5 * (a.x + b.x), (R)0.5 * (a.y + b.y));
        }
        __syncthreads();
        if (k + 3 < K) level_assemble<R, M>(md, pl, e, blk, k + 3, diag, W);
        // ---- L_{k+j,k} = W(k+j, k) D^-1
        cx<R>* X = sm;
        cx<R>* Y = sm + S2;
        for (int j = 1; j <= 2 && k + j < K; ++j) {
            __syncthreads();
            const cx<R>* A = slot(k + j, k);
            for (long long t = threadIdx.x; t < S2; t += blockDim.x) {
                const int r = (int)(t / S), c = (int)(t - (long long)r * S);
                X[t] = A[t];
                Y[t] = Dt[(long long)c * S + r];
            }
            __syncthreads();
            cx<R>* Lb = out(k, 2 + j);
            cx<R>* Lf = out(k + j, j);
            level_gemm<R>(S, X, Y, [&](int r, int c, cx<R> v) {
                Lb[(long long)r * S + c] = v;
                Lf[(long long)c * S + r] = v;
            });
        }
        // ---- Schur complements W(k+i, k+j) -= L_{k+i,k} W(k+j, k)^T
        for (int i = 1; i <= 2 && k + i < K; ++i)
            for (int j = 1; j <= i; ++j) {
                __syncthreads();
                const cx<R>* A = out(k, 2 + i);
                const cx<R>* B = slot(k + j, k);
                for (long long t = threadIdx.x; t < S2; t += blockDim.x) {
                    const int r = (int)(t / S), c = (int)(t - (long long)r * S);
                    X[t] = A[t];
                    Y[(long long)c * S + r] = B[t];
                }
                __syncthreads();
                cx<R>* C = slot(k + i, k + j);
                level_gemm<R>(S, X, Y, [&](int r, int c, cx<R> v) {
                    C[(long long)r * S + c] = csub<R>(C[(long long)r * S + c], v);
                });
            }
    }
    __syncthreads();
    if (threadIdx.x == 0 && bad_sh) atomicExch(fail + e, 1);
}

// z = B^-1 r for the level-blocked factors: one CTA per (selected system, block) of
// 4 * RW threads (grid: systems x blocks, systems fastest, so that the systems sharing an
// energy read each block's factors while they are in L2), RW = 32 ceil(S / 32): thread (q, i) sums quarter q of the inner index for row
// i of every level block product (4 x more loads in flight than one thread per row), and
// quarter 0 combines.  Forward: w_k = r_k - sum_j L_{k,k-j} w_{k-j}, u_k = D_k^-1 w_k (stored
// in z); backward: z_k = u_k - sum_j L_{k+j,k}^T z_{k+j}.  Optional partials
// part[s * nblk + blk] = sum_k w_k^T u_k (= r^T z restricted to the block).
constexpr int LA_RWMAX = 96;  // rows per quarter (>= LV_SMAX, a multiple of 32)
template <class R>
__global__ void __launch_bounds__(4 * LA_RWMAX) k_level_apply(PlanDev pl, const int* __restrict__ sys_e, Sel sel,
                                                             const cx<R>* __restrict__ F, const cx<R>* __restrict__ r,
                                                             long long rs, cx<R>* __restrict__ z, long long zs,
                                                             double2* __restrict__ part) {
    __shared__ cx<R> ring[3][LA_RWMAX];
    __shared__ cx<R> red[4][LA_RWMAX];   // partials of w (forward) and z (backward)
    __shared__ cx<R> redu[4][LA_RWMAX];  // partials of u: quarter 0 may still read them while
                                         // the next level's w partials are written
    __shared__ cx<R> sh[32];
    const int s = sel.list ? sel.list[blockIdx.x] : (int)blockIdx.x;
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const int S = pl.S, K = pl.K, L = pl.L, blk = blockIdx.y;
    const int RW = blockDim.x >> 2, i = threadIdx.x % RW, q = threadIdx.x / RW;
    const int Q = S >> 2, m0 = q * Q;  // this thread's quarter of the inner index
    const long long S2 = (long long)S * S;
    const int e = sys_e[s];
    const cx<R>* Out = F + (long long)e * level_factor_entries(pl.nblk, K, S) + (long long)blk * K * 5 * S2;
    const cx<R>* rv = r + (long long)s * rs;
    cx<R>* zv = z + (long long)s * zs;
    const int base = pl.fixed_base[blk];
    const bool row = i < S;
    cx<R> rz = mkc<R>(0, 0);
    // partial sum over this quarter of M[m][i] v[m] (M row-major S x S, v in shared memory)
    auto quarter = [&](const cx<R>* M, const cx<R>* v, cx<R> acc) {
        const cx<R>* col = M + (long long)m0 * S + i;
#pragma unroll 10
        for (int m = 0; m < Q; ++m) acc = cfma<R>(col[(long long)m * S], v[m0 + m], acc);
        return acc;
    };
    for (int k = 0; k < K; ++k) {
        const int c = k * S + i;
        const bool valid = row && q == 0 && c < L;
        const int el = valid ? base + pl.chain_off[c] : 0;
        const cx<R> rk = valid ? rv[el] : mkc<R>(0, 0);
        cx<R> part_w = mkc<R>(0, 0);
        if (row)
            for (int j = 1; j <= 2 && k - j >= 0; ++j)
                part_w = quarter(Out + ((long long)k * 5 + j) * S2, ring[(k - j) % 3], part_w);
        red[q][i] = part_w;
        __syncthreads();
        cx<R> w = mkc<R>(0, 0);
        if (row && q == 0) {
            w = csub<R>(csub<R>(csub<R>(csub<R>(rk, red[0][i]), red[1][i]), red[2][i]), red[3][i]);
            ring[k % 3][i] = w;
        }
        __syncthreads();
        cx<R> part_u = mkc<R>(0, 0);
        if (row) part_u = quarter(Out + (long long)k * 5 * S2, ring[k % 3], part_u);
        redu[q][i] = part_u;
        __syncthreads();
        if (row && q == 0) {
            const cx<R> u = cadd<R>(cadd<R>(cadd<R>(redu[0][i], redu[1][i]), redu[2][i]), redu[3][i]);
            rz = cfma<R>(w, u, rz);
            if (valid) zv[el] = u;
        }
    }
    __syncthreads();
    for (int k = K - 1; k >= 0; --k) {
        const int c = k * S + i;
        const bool valid = row && q == 0 && c < L;
        const int el = valid ? base + pl.chain_off[c] : 0;
        const cx<R> uk = valid ? zv[el] : mkc<R>(0, 0);
        cx<R> part_z = mkc<R>(0, 0);
        if (row)
            for (int j = 1; j <= 2 && k + j < K; ++j)
                part_z = quarter(Out + ((long long)k * 5 + 2 + j) * S2, ring[(k + j) % 3], part_z);
        red[q][i] = part_z;
        __syncthreads();
        if (row && q == 0) {
            const cx<R> zk = csub<R>(csub<R>(csub<R>(csub<R>(uk, red[0][i]), red[1][i]), red[2][i]), red[3][i]);
            ring[k % 3][i] = zk;
            if (valid) zv[el] = zk;
        }
        __syncthreads();
    }
    if (part) {
        const double2 tot = block_sum_c<R>(rz, sh);
        if (threadIdx.x == 0) part[(long long)s * pl.nblk + blk] = tot;
    }
}

// Point preconditioners: mode 0 -> z = r / diag (Jacobi), mode -1 -> z = r.  Optional r^T z.
template <class R>
__global__ void __launch_bounds__(TPB) k_point_precond(int N, const int* __restrict__ sys_e, Sel sel,
                                                      int mode, const cx<R>* __restrict__ diag, const cx<R>* __restrict__ r,
                                                      long long rs, cx<R>* __restrict__ z, long long zs,
                                                      double2* __restrict__ part) {
    __shared__ cx<R> sh[32];
    const int s = sel_sys(sel);
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    cx<R> loc = mkc<R>(0, 0);
    if (i < N) {
        const cx<R> ri = r[(long long)s * rs + i];
        cx<R> zi = ri;
        if (mode == 0) zi = cdiv<R>(ri, diag[(long long)sys_e[s] * N + i]);
        z[(long long)s * zs + i] = zi;
        loc = cmul<R>(ri, zi);
    }
    if (part) {
        const double2 tot = block_sum_c<R>(loc, sh);
        if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = tot;
    }
}

// ------------------------------------------------------------------- refinement (FP64)
// First outer step: r = b (x = 0), partial ||r||^2.
// ||b||^2 of every system: one thread block per system (grid: nsys), one partial each.  FP32
// accumulation: the stopping test needs ||b|| to ~1e-7 only.
__global__ void __launch_bounds__(TPB) k_rhs_norm(int N, const double2* __restrict__ b, double2* __restrict__ part) {
    __shared__ float2 sh[32];
    const int s = blockIdx.x;
    const double2* bs = b + (long long)s * N;
    float acc = 0.f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double2 v = bs[i];
        if ((__double_as_longlong(v.x) | __double_as_longlong(v.y)) != 0) {  // b is mostly zero
            const float fx = (float)v.x, fy = (float)v.y;
            acc = fmaf(fx, fx, fmaf(fy, fy, acc));
        }
    }
    const double2 tot = block_sum_c<float>(make_float2(acc, 0.f), sh);
    if (threadIdx.x == 0) part[s] = tot;
}

// Outer convergence test on the FP64 residual (stopping rule of Sec. III, true residual).
__global__ void k_outer_check(int nsys, SysState* __restrict__ st, int* __restrict__ outer, int* __restrict__ inner,
                              const double2* __restrict__ part, int nb, const double* __restrict__ bn2, int first,
                              double tol, double inner_tol, int max_refine, int max_iter, int inner_cap,
                              int stall_check, int* __restrict__ count, int* __restrict__ olist,
                              int* __restrict__ ilist) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    inner[s] = 0;
    if (!outer[s]) return;
    double rr = 0.0;
    if (bn2) {  // first check with ||b||^2 known from the right-hand-side builder
        rr = bn2[s];
    } else {
        for (int k = 0; k < nb; ++k) rr += part[(long long)s * nb + k].x;
    }
    const double rn = sqrt(rr);
    SysState& S = st[s];
    if (first) {
        S.bnorm = rn;
        if (rn == 0.0) {
            S.status = VBK_SYS_ZERO_RHS;
            S.rnorm = 0.0;
            outer[s] = 0;
            return;
        }
    } else {
        S.refines += 1;
    }
    const double prev = S.rnorm;
    S.rnorm = rn;
    if (!isfinite(rn)) {
        S.status = VBK_SYS_NAN;
        outer[s] = 0;
        return;
    }
    if (rn <= tol * S.bnorm) {
        S.status = VBK_SYS_CONVERGED;
        outer[s] = 0;
        return;
    }
    if (stall_check && !first && !(rn <= 0.9 * prev)) {  // the inner FP32 solve no longer helps
        S.status = VBK_SYS_STALLED;
        outer[s] = 0;
        return;
    }
    if (S.refines >= max_refine || S.iters >= max_iter) {
        S.status = VBK_SYS_MAX_ITER;
        outer[s] = 0;
        return;
    }
    S.pscale = S.scale;
    S.scale = rn;
    S.inv_scale = 1.0 / rn;
    S.target = fmax(inner_tol, 0.3 * tol * S.bnorm / rn);
    S.j = 0;
    S.last_cycle = S.cycle_iters;
    S.cycle_iters = 0;
    // the inner solve ends at max_iter, or after inner_cap iterations (the FP64 residual then
    // restarts it: a cure for FP32 Krylov stagnation)
    S.icap = inner_cap > 0 ? (int)min((long long)max_iter, (long long)S.iters + inner_cap) : max_iter;
    S.inres = 1.0;
    inner[s] = 1;
    const int pos = atomicAdd(count, 1);
    olist[pos] = s;
    ilist[pos] = s;
}

// inner right-hand side r / ||r|| in the inner precision
// Reorders the outer and inner lists of the next inner solve, longest expected solve first:
// one CTA per system runs the whole inner solve in the resident kernel, and the hardware
// starts CTAs in list order, so a long system started last leaves the other SMs idle.  Key:
// iterations of the system's previous inner solve, then the system index (later first: in an
// ascending energy grid, the higher energies with more open channels take longer), both
// descending.  One CTA; rank by counting (the caller limits this to ORDER_MAX systems).
constexpr int ORDER_MAX = 4096;
__global__ void __launch_bounds__(1024) k_order_lists(int nsys, const SysState* __restrict__ st, const int* __restrict__ inner,
                                                      int* __restrict__ olist, int* __restrict__ ilist) {
    __shared__ int key[ORDER_MAX];
    for (int s = threadIdx.x; s < nsys; s += blockDim.x) key[s] = inner[s] ? st[s].last_cycle : -1;
    __syncthreads();
    for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
        const int ks = key[s];
        if (ks < 0) continue;
        int pos = 0;
        for (int t = 0; t < nsys; ++t) {
            const int kt = key[t];
            pos += (kt > ks) || (kt == ks && t > s);
        }
        olist[pos] = s;
        ilist[pos] = s;
    }
}

template <class R>
__global__ void __launch_bounds__(TPB) k_inner_rhs(int N, Sel sel, const SysState* __restrict__ st,
                                                  const double2* __restrict__ r, cx<R>* __restrict__ out, long long os) {
    const int s = sel_sys(sel);
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 v = r[(long long)s * N + i];
    if constexpr (sizeof(R) == 4) {
        // narrow first, scale in FP32: no FP64 arithmetic per element
        const float inv = (float)st[s].inv_scale;
        out[(long long)s * os + i] = make_float2((float)v.x * inv, (float)v.y * inv);
    } else {
        const double inv = st[s].inv_scale;
        out[(long long)s * os + i] = cvt_from_d<R>(make_double2(v.x * inv, v.y * inv));
    }
}

// x += ||r|| d (FP64 accumulation of the inner correction)
template <class R>
__global__ void __launch_bounds__(TPB) k_accumulate(int N, Sel sel, const SysState* __restrict__ st,
                                                   const cx<R>* __restrict__ dv, long long ds, double2* __restrict__ x) {
    const int s = sel_sys(sel);
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double sc = st[s].scale;
    const double2 v = cvt_to_d<R>(dv[(long long)s * ds + i]);
    double2 xv = x[(long long)s * N + i];
    xv.x += sc * v.x;
    xv.y += sc * v.y;
    x[(long long)s * N + i] = xv;
}

// ----------------------------------------------------------------------------- COCG
// Two-term preconditioned COCG (Sec. III.A; van der Vorst & Melissen):
//   q = A p; alpha = rho / p^T q; x += alpha p; r -= alpha q; z = B^-1 r; rho' = r^T z;
//   beta = rho'/rho; p = z + beta p.
// rho = r^T z of a new inner solve.  With `cont` the search direction of the previous inner
// solve carries over (a reliable update: the recursive residual has just been replaced by the
// true FP64 residual): p = z + gamma p_old with gamma = (rho / rho_old) (scale / scale_old),
// the COCG beta of the unscaled recurrences expressed in the new inner scale; gamma = 0 starts
// afresh (p = z).
__global__ void k_cocg_start(int nsys, SysState* __restrict__ st, const int* __restrict__ act,
                             const double2* __restrict__ part_rz, int nb, int cont) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || !act[s]) return;
    double2 rz = make_double2(0.0, 0.0);
    for (int k = 0; k < nb; ++k) {
        rz.x += part_rz[(long long)s * nb + k].x;
        rz.y += part_rz[(long long)s * nb + k].y;
    }
    SysState& S = st[s];
    double2 g = make_double2(0.0, 0.0);
    const double den = S.rho.x * S.rho.x + S.rho.y * S.rho.y;
    if (cont && S.pscale > 0.0 && den > 0.0 && isfinite(den)) {
        g = cdiv<double>(rz, S.rho);
        const double f = S.scale / S.pscale;
        g.x *= f;
        g.y *= f;
        if (!isfinite(g.x) || !isfinite(g.y)) g = make_double2(0.0, 0.0);
    }
    S.rho = rz;
    S.beta = g;
}

// per-system scalars: one warp per system sums its partials (lanes strided, then shuffles)
__device__ __forceinline__ double2 warp_psum(const double2* __restrict__ p, int n) {
    const int lane = threadIdx.x & 31;
    double2 a = make_double2(0.0, 0.0);
    for (int k = lane; k < n; k += 32) {
        a.x += p[k].x;
        a.y += p[k].y;
    }
    return warp_sum2(a);  // valid in lane 0
}

__global__ void k_cocg_alpha(int nsys, SysState* __restrict__ st, int* __restrict__ act, int* __restrict__ outer,
                             const double2* __restrict__ part, int nb) {
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= nsys || !act[s]) return;
    const double2 pq = warp_psum(part + (long long)s * nb, nb);
    if ((threadIdx.x & 31) != 0) return;
    SysState& S = st[s];
    const double den = pq.x * pq.x + pq.y * pq.y;
    if (!(den > 0.0) || !isfinite(den)) {
        S.status = isfinite(den) ? VBK_SYS_BREAKDOWN : VBK_SYS_NAN;
        S.alpha = make_double2(0.0, 0.0);
        act[s] = 0;
        outer[s] = 0;
        return;
    }
    S.alpha = cdiv<double>(S.rho, pq);
}

template <class R>
__global__ void __launch_bounds__(TPB) k_cocg_update(int N, Sel sel, const SysState* __restrict__ st,
                                                    const int* __restrict__ sys_e, int pmode, const cx<R>* __restrict__ diag,
                                                    cx<R>* __restrict__ x, cx<R>* __restrict__ r, const cx<R>* __restrict__ p,
                                                    const cx<R>* __restrict__ q, cx<R>* __restrict__ z,
                                                    double2* __restrict__ part_rr, double2* __restrict__ part_rz) {
    __shared__ cx<R> sh[32];
    const int s = sel_sys(sel);
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    cx<R> lrr = mkc<R>(0, 0), lrz = mkc<R>(0, 0);
    if (i < N) {
        const long long o = (long long)s * N + i;
        const cx<R> al = cvt_from_d<R>(st[s].alpha);
        x[o] = cfma<R>(al, p[o], x[o]);
        const cx<R> qa = cmul<R>(al, q[o]);
        const cx<R> rn = csub<R>(r[o], qa);
        r[o] = rn;
        lrr.x = cabs2<R>(rn);
        if (pmode <= 0) {
            const cx<R> zi = pmode == 0 ? cdiv<R>(rn, diag[(long long)sys_e[s] * N + i]) : rn;
            z[o] = zi;
            lrz = cmul<R>(rn, zi);
        }
    }
    double2 tot = block_sum_c<R>(lrr, sh);
    if (threadIdx.x == 0) part_rr[(long long)s * gridDim.x + blockIdx.x] = tot;
    if (pmode <= 0) {
        tot = block_sum_c<R>(lrz, sh);
        if (threadIdx.x == 0) part_rz[(long long)s * gridDim.x + blockIdx.x] = tot;
    }
}

__global__ void k_cocg_beta(int nsys, SysState* __restrict__ st, int* __restrict__ act, int* __restrict__ outer,
                            const double2* __restrict__ part_rr, int nb_rr, const double2* __restrict__ part_rz, int nb_rz,
                            int max_iter, int* __restrict__ count, int* __restrict__ ilist) {
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= nsys || !act[s]) return;
    const double rr = warp_psum(part_rr + (long long)s * nb_rr, nb_rr).x;
    const double2 rz = warp_psum(part_rz + (long long)s * nb_rz, nb_rz);
    if ((threadIdx.x & 31) != 0) return;
    SysState& S = st[s];
    S.iters += 1;
    S.cycle_iters += 1;
    const double rn = sqrt(rr);
    S.inres = rn;
    if (!isfinite(rn) || !isfinite(rz.x) || !isfinite(rz.y)) {
        act[s] = 0;  // the outer FP64 residual decides (a NaN there ends the system)
        return;
    }
    if (rn <= S.target || S.iters >= S.icap) {
        act[s] = 0;
        return;
    }
    const double den = S.rho.x * S.rho.x + S.rho.y * S.rho.y;
    if (!(rz.x * rz.x + rz.y * rz.y > 0.0) || !(den > 0.0)) {
        S.status = VBK_SYS_BREAKDOWN;
        act[s] = 0;
        outer[s] = 0;
        return;
    }
    S.beta = cdiv<double>(rz, S.rho);
    S.rho = rz;
    ilist[atomicAdd(count, 1)] = s;
}

template <class R>
__global__ void __launch_bounds__(TPB) k_cocg_p(int N, Sel sel, const SysState* __restrict__ st,
                                               const cx<R>* __restrict__ z, cx<R>* __restrict__ p) {
    const int s = sel_sys(sel);
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long o = (long long)s * N + i;
    const cx<R> be = cvt_from_d<R>(st[s].beta);
    p[o] = cfma<R>(be, p[o], z[o]);
}


// ------------------------------------------------ persistent COCG (point preconditioners)
// Grid-stride kernels over work items drawn from a device-side list of active systems, so the
// grids are static and one CUDA graph serves a whole solve.  The per-system scalar steps run in
// the last work item of each system (its partials are complete once the per-system counter
// `done` reaches the item count; the writer side fences before counting), so an iteration is
// three launches: matvec (+ alpha), update (+ beta, convergence, next list), p update.
struct DList {
    const int* list;
    const int* count;
};

// Sum n partials of one system with the lanes of one warp (L2 reads; the writers fenced).
__device__ __forceinline__ double2 warp_psum_cg(const double2* p, int n) {
    const int lane = threadIdx.x & 31;
    double2 a = make_double2(0.0, 0.0);
    for (int k = lane; k < n; k += 32) {
        const double2 v = __ldcg(p + k);
        a.x += v.x;
        a.y += v.y;
    }
    return warp_sum2(a);
}

// one matvec work item: S systems x EPT*TPB elements of state d (register-blocked, as k_matvec3)
template <class R, int S, int EPT>
__device__ __forceinline__ void pmatvec_item(const DevModel& md, const int* sys_e, const int* sy, int d, int nu0,
                                             const int* offs, int np, const cx<R>* diag, const cx<R>* x, cx<R>* y,
                                             cx<R> (&loc)[S]) {
    const int Nnu = md.Nnu, N = md.N;
    const int nv = min(EPT, Nnu - nu0);
    const int i0 = d * Nnu + nu0;
    const cx<R>* xp[S];
    cx<R> acc[S][EPT], xi[S][EPT];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        xp[t] = x + (long long)(sy[t] < 0 ? 0 : sy[t]) * N;
        const cx<R>* dg = diag + (long long)sys_e[sy[t] < 0 ? 0 : sy[t]] * N;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            xi[t][e] = mkc<R>(0, 0);
            acc[t][e] = mkc<R>(0, 0);
            if (sy[t] >= 0 && e < nv) {
                xi[t][e] = xp[t][i0 + e];
                acc[t][e] = cmul<R>(dg[i0 + e], xi[t][e]);
            }
        }
    }
    if (nv > 0) {
        // stencil points in batches of PB: all coefficient and neighbour loads of a batch are
        // issued before its FMAs (memory-level parallelism; short critical path)
        constexpr int PB = 4;
        const R* pc = pcp<R>(md) + (long long)md.ebeg[d] * Nnu + nu0;
        const bool interior = nv == EPT;
        for (int k0 = 0; k0 < np; k0 += PB) {
            R c[PB][EPT];
            cx<R> v[PB][S][EPT];
#pragma unroll
            for (int kk = 0; kk < PB; ++kk) {
                const int k = k0 + kk;
                const bool okk = k < np;
                const int j0 = i0 + (okk ? offs[k] : 0);
                const bool fast = interior && j0 >= 0 && j0 + EPT <= N;
#pragma unroll
                for (int e = 0; e < EPT; ++e) c[kk][e] = (okk && e < nv) ? __ldg(pc + (long long)k * Nnu + e) : (R)0;
#pragma unroll
                for (int t = 0; t < S; ++t)
#pragma unroll
                    for (int e = 0; e < EPT; ++e) {
                        const int j = fast ? j0 + e : min(max(j0 + e, 0), N - 1);
                        v[kk][t][e] = xp[t][j];
                    }
            }
#pragma unroll
            for (int kk = 0; kk < PB; ++kk)
#pragma unroll
                for (int t = 0; t < S; ++t)
#pragma unroll
                    for (int e = 0; e < EPT; ++e) {
                        acc[t][e].x = fma(-c[kk][e], v[kk][t][e].x, acc[t][e].x);
                        acc[t][e].y = fma(-c[kk][e], v[kk][t][e].y, acc[t][e].y);
                    }
        }
    }
#pragma unroll
    for (int t = 0; t < S; ++t) {
        loc[t] = mkc<R>(0, 0);
        if (sy[t] < 0) continue;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            if (e >= nv) continue;
            y[(long long)sy[t] * N + i0 + e] = acc[t][e];
            loc[t] = cfma<R>(xi[t][e], acc[t][e], loc[t]);
        }
    }
}

// q = A p and p^T q; the last item of a system sets alpha = rho / p^T q (breakdown: retire).
template <class R, int S, int EPT>
__global__ void __launch_bounds__(TPB) k_pmatvec(DevModel md, const int* __restrict__ sys_e, DList L,
                                                const cx<R>* __restrict__ diag, const cx<R>* __restrict__ p,
                                                cx<R>* __restrict__ q, double2* __restrict__ part, int* __restrict__ done,
                                                SysState* __restrict__ st, int* __restrict__ act, int* __restrict__ outer) {
    __shared__ int offs[MAXS][MV_MAXPTS];
    __shared__ cx<R> redsh[TPB / 32][S];
    __shared__ int lastf[S];
    constexpr int T = TPB * EPT;
    const int Nnu = md.Nnu;
    const int nchunk = (Nnu + T - 1) / T;
    const int nxb = md.ns * nchunk;  // items (and partials) per system group
    for (int dd = 0; dd < md.ns; ++dd) {
        const int pb = md.ebeg[dd], np = min(md.ebeg[dd + 1] - pb, MV_MAXPTS);
        for (int k = threadIdx.x; k < np; k += blockDim.x) {
            const DevEntry& e = md.ent[pb + k];
            offs[dd][k] = (e.dp - dd) * Nnu + e.lin;
        }
    }
    __syncthreads();
    const int cnt = *L.count;
    const int ngr = (cnt + S - 1) / S;
    const int nitems = ngr * nxb;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int g = item / nxb, xb = item - g * nxb;
        const int d = xb / nchunk;
        const int nu0 = (xb - d * nchunk) * T + threadIdx.x * EPT;
        int sy[S];
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const int pos = g * S + t;
            sy[t] = pos < cnt ? L.list[pos] : -1;
        }
        const int np = min(md.ebeg[d + 1] - md.ebeg[d], MV_MAXPTS);
        cx<R> loc[S];
        pmatvec_item<R, S, EPT>(md, sys_e, sy, d, nu0, offs[d], np, diag, p, q, loc);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const cx<R> v = warp_sum_c<R>(loc[t]);
            if (lane == 0) redsh[w][t] = v;
        }
        __syncthreads();
        if (threadIdx.x < S) {
            const int t = threadIdx.x, sid = sy[t];
            lastf[t] = 0;
            if (sid >= 0) {
                cx<R> tot = mkc<R>(0, 0);
                for (int qq = 0; qq < TPB / 32; ++qq) tot = cadd<R>(tot, redsh[qq][t]);
                part[(long long)sid * nxb + xb] = cvt_to_d<R>(tot);
                __threadfence();
                lastf[t] = atomicAdd(done + sid, 1) == nxb - 1;
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < S; ++t) {
            if (!lastf[t]) continue;  // uniform across the block
            if (w == 0) {
                __threadfence();
                const int sid = sy[t];
                const double2 pq = warp_psum_cg(part + (long long)sid * nxb, nxb);
                if (lane == 0) {
                    done[sid] = 0;
                    SysState& Sx = st[sid];
                    const double den = pq.x * pq.x + pq.y * pq.y;
                    if (!(den > 0.0) || !isfinite(den)) {
                        Sx.status = isfinite(den) ? VBK_SYS_BREAKDOWN : VBK_SYS_NAN;
                        Sx.alpha = make_double2(0.0, 0.0);
                        act[sid] = 0;
                        outer[sid] = 0;
                    } else {
                        Sx.alpha = cdiv<double>(Sx.rho, pq);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// x += alpha p, r -= alpha q, z = B^-1 r (point), partials ||r||^2 and r^T z; the last item of a
// system forms beta, tests convergence and appends the system to the next list.
template <class R, int EPT>
__global__ void __launch_bounds__(TPB) k_pupdate(int N, const int* __restrict__ sys_e, DList L, int pmode,
                                                const cx<R>* __restrict__ diag, cx<R>* __restrict__ x, cx<R>* __restrict__ r,
                                                const cx<R>* __restrict__ p, const cx<R>* __restrict__ q, cx<R>* __restrict__ z,
                                                double2* __restrict__ part_rr, double2* __restrict__ part_rz,
                                                int* __restrict__ done, SysState* __restrict__ st, int* __restrict__ act,
                                                int* __restrict__ outer, int max_iter, int* __restrict__ next_list,
                                                int* __restrict__ next_count) {
    __shared__ R red3[TPB / 32][3];
    __shared__ int lastf;
    constexpr int T = TPB * EPT;
    const int nub = (N + T - 1) / T;
    const int cnt = *L.count;
    const int nitems = cnt * nub;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int pos = item / nub, ub = item - pos * nub;
        const int s = L.list[pos];
        const bool on = act[s] != 0;  // a breakdown in this iteration's matvec retired it
        cx<R> lrr = mkc<R>(0, 0), lrz = mkc<R>(0, 0);
        if (on) {
            const cx<R> al = cvt_from_d<R>(st[s].alpha);
            const long long so = (long long)s * N;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const int i = ub * T + e * TPB + threadIdx.x;
                if (i >= N) continue;
                const long long o = so + i;
                x[o] = cfma<R>(al, p[o], x[o]);
                const cx<R> rn = csub<R>(r[o], cmul<R>(al, q[o]));
                r[o] = rn;
                lrr.x += cabs2<R>(rn);
                const cx<R> zi = pmode == 0 ? cdiv<R>(rn, diag[(long long)sys_e[s] * N + i]) : rn;
                z[o] = zi;
                lrz = cfma<R>(rn, zi, lrz);
            }
        }
        // one block reduction of (||r||^2, r^T z)
        R a0 = lrr.x, a1 = lrz.x, a2 = lrz.y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_down_sync(0xffffffffu, a0, o);
            a1 += __shfl_down_sync(0xffffffffu, a1, o);
            a2 += __shfl_down_sync(0xffffffffu, a2, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red3[threadIdx.x >> 5][0] = a0;
            red3[threadIdx.x >> 5][1] = a1;
            red3[threadIdx.x >> 5][2] = a2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            lastf = 0;
            if (on) {
                R b0 = 0, b1 = 0, b2 = 0;
                for (int w = 0; w < TPB / 32; ++w) {
                    b0 += red3[w][0];
                    b1 += red3[w][1];
                    b2 += red3[w][2];
                }
                part_rr[(long long)s * nub + ub] = make_double2((double)b0, 0.0);
                part_rz[(long long)s * nub + ub] = make_double2((double)b1, (double)b2);
                __threadfence();
                lastf = atomicAdd(done + s, 1) == nub - 1;
            }
        }
        __syncthreads();
        if (lastf && threadIdx.x < 32) {
            __threadfence();
            const double rr = warp_psum_cg(part_rr + (long long)s * nub, nub).x;
            const double2 rz = warp_psum_cg(part_rz + (long long)s * nub, nub);
            if (threadIdx.x == 0) {
                done[s] = 0;
                SysState& Sx = st[s];
                Sx.iters += 1;
                Sx.cycle_iters += 1;
                const double rn = sqrt(rr);
                Sx.inres = rn;
                const double den = Sx.rho.x * Sx.rho.x + Sx.rho.y * Sx.rho.y;
                if (!isfinite(rn) || !isfinite(rz.x) || !isfinite(rz.y) || rn <= Sx.target || Sx.iters >= Sx.icap) {
                    act[s] = 0;  // the FP64 residual decides
                } else if (!(rz.x * rz.x + rz.y * rz.y > 0.0) || !(den > 0.0)) {
                    Sx.status = VBK_SYS_BREAKDOWN;
                    act[s] = 0;
                    outer[s] = 0;
                } else {
                    Sx.beta = cdiv<double>(rz, Sx.rho);
                    Sx.rho = rz;
                    next_list[atomicAdd(next_count, 1)] = s;
                }
            }
        }
        __syncthreads();
    }
}

// p = z + beta p for the systems of the next list
template <class R, int EPT>
__global__ void __launch_bounds__(TPB) k_pp(int N, DList L, const SysState* __restrict__ st, const cx<R>* __restrict__ z,
                                           cx<R>* __restrict__ p) {
    constexpr int T = TPB * EPT;
    const int nub = (N + T - 1) / T;
    const int cnt = *L.count;
    const int nitems = cnt * nub;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int pos = item / nub, ub = item - pos * nub;
        const int s = L.list[pos];
        const cx<R> be = cvt_from_d<R>(st[s].beta);
        const long long so = (long long)s * N;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int i = ub * T + e * TPB + threadIdx.x;
            if (i < N) p[so + i] = cfma<R>(be, p[so + i], z[so + i]);
        }
    }
}


// --------------------------------------------------- resident COCG (one CTA per system)
// The whole inner solve of one system runs in one CTA: p and q live in shared memory (q is
// overwritten by z = B^-1 r once consumed), x, r and the diagonal table stay in global memory
// (L2-resident for the systems in flight), and the scalars come from block reductions.  No
// grid-wide synchronisation is needed because the systems are independent; a converged system
// frees its SM for the next one.  The iteration count is bounded by max_iter.

// r = b - A x for the FP32 refinement path in double-float arithmetic.  x, r and the diagonal
// are (re hi, im hi, re lo, im lo) quadruples, b is FP64 (split where nonzero); the energy-independent stencil
// coefficients come as (hi, lo) pairs.  Register blocking as in k_matvec3 (S systems x EPT
// consecutive elements per thread, coefficients loaded once for the S systems); one
// ||r||^2 partial (of the hi parts: FP32 within a warp, FP64 across warps) per thread block and system.
template <int S, int EPT>
__global__ void __launch_bounds__(TPB) k_residual_df(DevModel md, const int* __restrict__ sys_e, Sel sel, int nlist,
                                                    const float4* __restrict__ dsp, const float4* __restrict__ xs,
                                                    const double2* __restrict__ b64, float4* __restrict__ rs,
                                                    double2* __restrict__ part) {
    __shared__ int offs[MV_MAXPTS];
    __shared__ double redsh[TPB / 32][S];
    constexpr int T = TPB * EPT;
    const int Nnu = md.Nnu, N = md.N;
    const int nchunk = (Nnu + T - 1) / T;
    const int d = blockIdx.x / nchunk;
    const int nu0 = (blockIdx.x - d * nchunk) * T + threadIdx.x * EPT;
    const int pb = md.ebeg[d], np = min(md.ebeg[d + 1] - pb, MV_MAXPTS);
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const DevEntry& e = md.ent[pb + k];
        offs[k] = (e.dp - d) * Nnu + e.lin;
    }
    int sy[S];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const int li = blockIdx.y * S + t;
        int s = -1;
        if (li < nlist) {
            s = sel.list ? sel.list[li] : li;
            if (s >= 0 && sel.act && !sel.act[s]) s = -1;
        }
        sy[t] = s;
    }
    __syncthreads();
    const int nv = min(EPT, Nnu - nu0);
    const int i0 = d * Nnu + nu0;
    float rh[S][EPT], rl[S][EPT], ih[S][EPT], il[S][EPT];  // r = (rh + rl) + i (ih + il)
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const long long so = (long long)(sy[t] < 0 ? 0 : sy[t]) * N;
        const float4* dg = dsp + (long long)sys_e[sy[t] < 0 ? 0 : sy[t]] * N;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            rh[t][e] = rl[t][e] = ih[t][e] = il[t][e] = 0.f;
            if (sy[t] >= 0 && e < nv) {
                const float4 x = xs[so + i0 + e], g = dg[i0 + e];
                const double2 b = b64[so + i0 + e];
                if ((__double_as_longlong(b.x) | __double_as_longlong(b.y)) != 0) {  // b is mostly zero
                    rh[t][e] = (float)b.x;
                    ih[t][e] = (float)b.y;
                    rl[t][e] = (float)(b.x - (double)rh[t][e]);
                    il[t][e] = (float)(b.y - (double)ih[t][e]);
                }
                df_fma(rh[t][e], rl[t][e], -g.x, -g.z, x.x, x.z);
                df_fma(rh[t][e], rl[t][e], g.y, g.w, x.y, x.w);
                df_fma(ih[t][e], il[t][e], -g.x, -g.z, x.y, x.w);
                df_fma(ih[t][e], il[t][e], -g.y, -g.w, x.x, x.z);
            }
        }
    }
    if (nv > 0) {
        const float2* pc = md.pcs + (long long)pb * Nnu + nu0;
        for (int k = 0; k < np; ++k) {
            float2 c[EPT];
#pragma unroll
            for (int e = 0; e < EPT; ++e) c[e] = e < nv ? __ldg(pc + (long long)k * Nnu + e) : make_float2(0.f, 0.f);
            const int j0 = i0 + offs[k];
#pragma unroll
            for (int t = 0; t < S; ++t) {
                const float4* xb = xs + (long long)(sy[t] < 0 ? 0 : sy[t]) * N;
#pragma unroll
                for (int e = 0; e < EPT; ++e) {
                    const float4 v = xb[min(max(j0 + e, 0), N - 1)];  // zero coefficient outside the basis
                    df_fma(rh[t][e], rl[t][e], c[e].x, c[e].y, v.x, v.z);
                    df_fma(ih[t][e], il[t][e], c[e].x, c[e].y, v.y, v.w);
                }
            }
        }
    }
    float loc[S];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        loc[t] = 0.f;
        if (sy[t] < 0) continue;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            if (e >= nv) continue;
            const float2 re = df_norm(rh[t][e], rl[t][e]), im = df_norm(ih[t][e], il[t][e]);
            rs[(long long)sy[t] * N + i0 + e] = make_float4(re.x, im.x, re.y, im.y);
            loc[t] = fmaf(re.x, re.x, fmaf(im.x, im.x, loc[t]));
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < S; ++t) {
        float v = loc[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) redsh[w][t] = (double)v;  // FP32 within a warp, FP64 across warps
    }
    __syncthreads();
    if (threadIdx.x < S && sy[threadIdx.x] >= 0) {
        double tot = 0.0;
        for (int q = 0; q < TPB / 32; ++q) tot += redsh[q][threadIdx.x];
        part[(long long)sy[threadIdx.x] * gridDim.x + blockIdx.x] = make_double2(tot, 0.0);
    }
}
constexpr int DF_S = 2, DF_EPT = 4;
inline int df_partials(const DevModel& md) { return md.ns * ((md.Nnu + TPB * DF_EPT - 1) / (TPB * DF_EPT)); }


// x64 = hi + lo of the double-float solution (every system); the sum is exact in FP64.  Two
// entries per thread (independent loads in flight), streamed: neither side is read again here.
__global__ void __launch_bounds__(TPB) k_df_out(long long n, const float4* __restrict__ xs, double2* __restrict__ x64) {
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (i >= n) return;
    const bool two = i + 1 < n;
    const float4 v = __ldcs(xs + i);
    const float4 u = two ? __ldcs(xs + i + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    __stcs(x64 + i, make_double2(f2d_exact(v.x) + f2d_exact(v.z), f2d_exact(v.y) + f2d_exact(v.w)));
    if (two) __stcs(x64 + i + 1, make_double2(f2d_exact(u.x) + f2d_exact(u.z), f2d_exact(u.y) + f2d_exact(u.w)));
}

constexpr int RTPB = 1024;


// SEC: some stencil point involves a second mode (its factor from the oscillator tables); the
// instantiation without it drops that test from the point loop.
template <int M, bool SEC>
__global__ void __launch_bounds__(RTPB, 1) k_cocg_resident(DevModel md, const int* __restrict__ sys_e,
                                                          const int* __restrict__ list, int pmode,
                                                          const float2* __restrict__ diag, const float2* __restrict__ dinv,
                                                          float2* __restrict__ x, float2* __restrict__ r,
                                                          const double2* __restrict__ res_d, const float4* __restrict__ res_s,
                                                          float4* __restrict__ xs,
                                                          SysState* __restrict__ st, int* __restrict__ act,
                                                          int* __restrict__ outer, int max_iter) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = md.N, H = md.rhalo;
    float2* P = reinterpret_cast<float2*>(smraw) + H;  // p with H zero entries on either side
    float2* Q = P + N + H;
    float2* sct = Q + N;                                 // coefficient rows (packed pairs)
    __shared__ int4 sdesc[MAXS * 64];
    __shared__ float redA[RTPB / 32][3], redB[RTPB / 32][3];  // per-warp partials of the two reductions
    static_assert(RTPB == 1024, "one partial per lane in the final warp sums");
    const int s = list[blockIdx.x];
    if (s < 0) return;  // launched over more list slots than systems (speculative refinement round)
    const int tid = threadIdx.x;
    const long long so = (long long)s * N;
    const float2* dg = diag + (long long)sys_e[s] * N;
    const float2* di = dinv + (long long)sys_e[s] * N;
    for (int k = tid; k < md.nrct; k += RTPB) sct[k] = md.rct[k];
    for (int k = tid; k < H; k += RTPB) P[-1 - k] = P[N + k] = make_float2(0.f, 0.f);
    for (int k = tid; k < md.rbeg[md.ns]; k += RTPB) sdesc[k] = md.rdesc[k];
    // per-system scalars, kept identical in every thread: each reduction ends with one barrier
    // after which every warp sums the per-warp partials itself (no serial thread-0 section)
    // (fields read where they are needed: nothing of the state stays live across the loop)
    const float target2 = (float)(st[s].target * st[s].target);
    int iters = st[s].iters;
    const int icap = min(max_iter, st[s].icap);
    float rr = 0.f;
    int status = -1;  // -1: stopped normally (the FP64 residual decides)
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5;
    auto all_sum3 = [&](float (*buf)[3], float a0, float a1, float a2) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
            buf[wid][0] = a0;
            buf[wid][1] = a1;
            buf[wid][2] = a2;
        }
        __syncthreads();
        float3 t = make_float3(buf[lane][0], buf[lane][1], buf[lane][2]);  // RTPB / 32 == 32 partials
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
            t.z += __shfl_xor_sync(0xffffffffu, t.z, o);
        }
        return t;
    };
    // start of the inner solve: r = (b - A x) / scale in FP32 (the hi part of the double-float
    // residual, scaled in FP32), x = 0, z = B^-1 r, p = z, rho = r^T z
    float2 rho, beta = make_float2(0.f, 0.f);
    {
        const float inv = (float)st[s].inv_scale;
        float rz_x = 0.f, rz_y = 0.f;
        for (int i = tid; i < N; i += RTPB) {
            float2 rn = make_float2(0.f, 0.f);
            if (res_d) {  // the first residual: b (FP64, mostly zero)
                const double2 v = res_d[so + i];
                if ((__double_as_longlong(v.x) | __double_as_longlong(v.y)) != 0)
                    rn = make_float2((float)v.x * inv, (float)v.y * inv);
            } else {
                const float4 v = res_s[so + i];
                rn = make_float2(v.x * inv, v.y * inv);
            }
            r[so + i] = rn;
            const float2 zi = pmode == 0 ? cmul<float>(rn, di[i]) : rn;
            P[i] = zi;
            rz_x += rn.x * zi.x - rn.y * zi.y;
            rz_y += rn.x * zi.y + rn.y * zi.x;
        }
        const float3 t = all_sum3(redB, 0.f, rz_x, rz_y);
        rho = make_float2(t.y, t.z);
    }
    bool wrote_x = false;
    const int budget = max(0, icap - iters);
    // mixed-radix digits of this thread's first element and of the stride RTPB
    int d0, n0[MAXM], inc[MAXM], incd;
    {
        d0 = (int)fdiv((unsigned)tid, md.fd_nnu);
        decode<M>(md, tid - d0 * md.Nnu, n0);
        incd = (int)fdiv((unsigned)RTPB, md.fd_nnu);
        decode<M>(md, RTPB - incd * md.Nnu, inc);
    }
    for (int it = 0; it < budget; ++it) {
        // q = A p and p^T q
        float pq_x = 0.f, pq_y = 0.f;
        // (d, n) of element i, advanced by RTPB in the mixed radix (d, n_0, ..., n_{M-1}) with
        // one carry per digit instead of a division per digit
        int d = d0;
        int n[MAXM];
#pragma unroll
        for (int m = 0; m < MAXM; ++m) n[m] = n0[m];
        for (int i = tid; i < N; i += RTPB) {
            if (i != tid) {
                int c = 0;
#pragma unroll
                for (int m = M - 1; m >= 0; --m) {
                    int v = n[m] + inc[m] + c;
                    c = v >= md.nb[m];
                    n[m] = c ? v - md.nb[m] : v;
                }
                d += incd + c;
            }
            const float2 pi = P[i];
            float2 acc = cmul<float>(dg[i], pi);
            const char* Pi = reinterpret_cast<const char*>(P + i);
            int k = md.rbeg[d];
#pragma unroll
            for (int m = 0; m < M; ++m) {  // points grouped by primary mode: no per-point mode select
                const int kend = k + md.rcnt[d][m];
                const char* row = reinterpret_cast<const char*>(sct) + n[m] * 8;
#pragma unroll 4
                for (; k < kend; ++k) {
                    const int4 q = sdesc[k];
                    float2 cc = *reinterpret_cast<const float2*>(row + q.x);  // (-c, -c)
                    if constexpr (SEC) {
                        if (q.z >= 0) {
                            const float t = md.tab32[q.z + nsel<M>(n, q.w)];
                            cc.x *= t;
                            cc.y *= t;
                        }
                    }
                    // neighbours outside [0, N) read the zero halo
                    acc = ffma2(cc, *reinterpret_cast<const float2*>(Pi + q.y), acc);
                }
            }
            Q[i] = acc;
            pq_x += pi.x * acc.x - pi.y * acc.y;
            pq_y += pi.x * acc.y + pi.y * acc.x;
        }
        const float3 pq = all_sum3(redA, pq_x, pq_y, 0.f);
        const float den = pq.x * pq.x + pq.y * pq.y;
        if (!(den > 0.f) || !isfinite(den)) {
            status = isfinite(den) ? VBK_SYS_BREAKDOWN : VBK_SYS_NAN;
            break;
        }
        const float2 al = make_float2((rho.x * pq.x + rho.y * pq.y) / den, (rho.y * pq.x - rho.x * pq.y) / den);
        // x += alpha p, r -= alpha q, z = B^-1 r (into Q), ||r||^2, r^T z
        float rr_l = 0.f, rz_x = 0.f, rz_y = 0.f;
        for (int i = tid; i < N; i += RTPB) {
            const float2 pi = P[i], qi = Q[i];
            float2 xv = it == 0 ? make_float2(0.f, 0.f) : x[so + i];
            xv.x += al.x * pi.x - al.y * pi.y;
            xv.y += al.x * pi.y + al.y * pi.x;
            x[so + i] = xv;
            float2 rn = r[so + i];
            rn.x -= al.x * qi.x - al.y * qi.y;
            rn.y -= al.x * qi.y + al.y * qi.x;
            r[so + i] = rn;
            const float2 zi = pmode == 0 ? cmul<float>(rn, di[i]) : rn;
            Q[i] = zi;
            rr_l += rn.x * rn.x + rn.y * rn.y;
            rz_x += rn.x * zi.x - rn.y * zi.y;
            rz_y += rn.x * zi.y + rn.y * zi.x;
        }
        const float3 sums = all_sum3(redB, rr_l, rz_x, rz_y);
        wrote_x = true;
        iters += 1;
        rr = sums.x;
        if (!isfinite(sums.x) || !isfinite(sums.y) || !isfinite(sums.z) || sums.x <= target2 || iters >= icap) break;
        const float rden = rho.x * rho.x + rho.y * rho.y;
        if (!(sums.y * sums.y + sums.z * sums.z > 0.f) || !(rden > 0.f)) {
            status = VBK_SYS_BREAKDOWN;
            break;
        }
        beta = make_float2((sums.y * rho.x + sums.z * rho.y) / rden, (sums.z * rho.x - sums.y * rho.y) / rden);
        rho = make_float2(sums.y, sums.z);
        // p = z + beta p
        for (int i = tid; i < N; i += RTPB) {
            const float2 pi = P[i], zi = Q[i];
            P[i] = make_float2(zi.x + beta.x * pi.x - beta.y * pi.y, zi.y + beta.x * pi.y + beta.y * pi.x);
        }
        __syncthreads();
    }
    // the correction of this refinement step: x += scale d in double-float (each thread its own
    // elements; scale split once into hi + lo floats)
    if (wrote_x) {
        const double sc = st[s].scale;
        const float sh = (float)sc, sl = (float)(sc - (double)sh);
        for (int i = tid; i < N; i += RTPB) {
            const float2 dv = x[so + i];
            float4 X = xs[so + i];
            df_fma(X.x, X.z, sh, sl, dv.x, 0.f);
            df_fma(X.y, X.w, sh, sl, dv.y, 0.f);
            const float2 re = df_norm(X.x, X.z), im = df_norm(X.y, X.w);
            xs[so + i] = make_float4(re.x, im.x, re.y, im.y);
        }
    }
    if (tid == 0) {
        SysState& S = st[s];
        S.cycle_iters += iters - S.iters;
        S.iters = iters;
        S.inres = sqrt((double)rr);
        S.rho = make_double2(rho.x, rho.y);
        S.beta = make_double2(beta.x, beta.y);
        if (status >= 0) {
            S.status = status;
            outer[s] = 0;
        }
        act[s] = 0;
    }
}

// b - A x in double-float for one system per CTA (grid: the outer list; -1 entries return):
// the whole split solution (re hi, im hi, re lo, im lo) of the system is staged once in shared
// memory with a zero halo, so every x entry leaves L2/HBM once instead of once per stencil
// point; coefficients come from the (hi, lo) rows of the primary mode (models whose points
// involve a secondary mode use k_residual_df).  One ||r||^2 partial per system (part[s]).
template <int M>
__global__ void __launch_bounds__(RTPB, 1) k_residual_res(DevModel md, const int* __restrict__ sys_e,
                                                         const int* __restrict__ list, const float4* __restrict__ dsp,
                                                         const float4* __restrict__ xs, const double2* __restrict__ b64,
                                                         float4* __restrict__ rs, double2* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = md.N, H = md.rhalo;
    float4* X = reinterpret_cast<float4*>(smraw) + H;
    float2* rows = reinterpret_cast<float2*>(X + N + H);
    __shared__ int4 sdesc[MAXS * 64];
    __shared__ double red[RTPB / 32];
    const int s = list[blockIdx.x];
    if (s < 0) return;
    const int tid = threadIdx.x;
    const long long so = (long long)s * N;
    const float4* dg = dsp + (long long)sys_e[s] * N;
    for (int k = tid; k < md.nrct; k += RTPB) rows[k] = md.rctd[k];
    for (int k = tid; k < H; k += RTPB) X[-1 - k] = X[N + k] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = tid; k < md.rbeg[md.ns]; k += RTPB) sdesc[k] = md.rdesc[k];
    for (int i = tid; i < N; i += RTPB) X[i] = xs[so + i];
    __syncthreads();
    float nrm = 0.f;
    for (int i = tid; i < N; i += RTPB) {
        const int d = (int)fdiv((unsigned)i, md.fd_nnu), nu = i - d * md.Nnu;
        int n[MAXM];
        decode<M>(md, nu, n);
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        const double2 bb = b64[so + i];
        if ((__double_as_longlong(bb.x) | __double_as_longlong(bb.y)) != 0) {  // b is mostly zero
            rh = (float)bb.x;
            ih = (float)bb.y;
            rl = (float)(bb.x - (double)rh);
            il = (float)(bb.y - (double)ih);
        }
        const float4 x = X[i], g = dg[i];
        df_fma(rh, rl, -g.x, -g.z, x.x, x.z);
        df_fma(rh, rl, g.y, g.w, x.y, x.w);
        df_fma(ih, il, -g.x, -g.z, x.y, x.w);
        df_fma(ih, il, -g.y, -g.w, x.x, x.z);
        int k = md.rbeg[d];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int kend = k + md.rcnt[d][m];
            const float2* row = rows + n[m];
#pragma unroll 4
            for (; k < kend; ++k) {
                const int4 q = sdesc[k];
                const float2 c = row[q.x >> 3];
                const float4 v = X[i + (q.y >> 3)];  // neighbours outside [0, N) read the zero halo
                df_fma(rh, rl, c.x, c.y, v.x, v.z);
                df_fma(ih, il, c.x, c.y, v.y, v.w);
            }
        }
        const float2 re = df_norm(rh, rl), im = df_norm(ih, il);
        rs[so + i] = make_float4(re.x, im.x, re.y, im.y);
        nrm = fmaf(re.x, re.x, fmaf(im.x, im.x, nrm));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, o);
    if ((tid & 31) == 0) red[tid >> 5] = (double)nrm;  // FP32 within a warp, FP64 across warps
    __syncthreads();
    if (tid < 32) {
        double t = red[tid];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (tid == 0) part[s] = make_double2(t, 0.0);
    }
}
inline size_t residual_res_smem(const DevModel& md) {
    return (size_t)(md.N + 2 * md.rhalo) * sizeof(float4) + (size_t)md.nrct * sizeof(float2) + 16;
}
// Fused mixed-precision solve, one 1024-thread CTA per system and every refinement step in the
// same launch.  A persistent grid (one CTA per SM: the CTA holds p, q and the coefficient rows in
// shared memory) takes systems from a counter, highest index first (the higher energies of an
// ascending grid open more channels and take longer), and for each runs
//   r = b - A x in double-float arithmetic (x staged in shared memory, b and the diagonal from
//   global), ||r|| (FP32 within a warp, FP64 across warps), the stopping / stall / cap checks of
//   the refinement, the FP32 COCG inner solve of the resident kernel on r / ||r||, and
//   x += ||r|| d in double-float,
// then writes psi = hi + lo in FP64.  This replaces, for such systems, the host loop of separate
// residual, check, ordering and output launches.
// QD (models whose points involve one mode and whose second-fastest mode has a multiple of 4
// functions): the two stencil loops (the FP32 product and the double-float residual) take quads
// of elements, i0 + c S for c = 0..3 with S = nb[M-1] -- the same state and quanta but for
// n[M-2] = 4 b + c -- so that each point's descriptor and (fastest-mode) coefficient are read
// once for four elements; the residual runs on both halves of (re, im) pairs at once (packed
// FP32x2 double-float steps, bit-identical to the scalar ones).
template <int M, bool SEC, bool QD>
__global__ void __launch_bounds__(RTPB, 1) k_solve_resident(DevModel md, ClArgs a, float2* __restrict__ xw,
                                                           float2* __restrict__ rw, const float2* __restrict__ dinv) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = md.N, H = md.rhalo, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float2* P = reinterpret_cast<float2*>(smraw) + H;  // p with H zero entries on either side
    float2* Q = P + N + H;
    float4* XS = reinterpret_cast<float4*>(smraw) + H;  // the split solution during the residual
    const size_t rows_off = std::max((size_t)(2 * N + 2 * H) * 8, (size_t)(N + 2 * H) * 16);
    float2* rows = reinterpret_cast<float2*>(smraw + rows_off);  // rct (FP32 pass) or rctd (residual)
    // one bit per element: b_i != 0 (set in the first pass, which reads b whole; b is a few
    // entries of an entry channel, so the later passes load only those)
    unsigned* bmask = reinterpret_cast<unsigned*>(smraw + rows_off + (((size_t)md.nrct * 8 + 15) & ~(size_t)15));
    const int NW = (N + 31) >> 5;
    __shared__ int4 sdesc[MAXS * 64];
    __shared__ float redA[RTPB / 32][3], redB[RTPB / 32][3];
    __shared__ double redD[RTPB / 32];
    __shared__ int snext;
    // per-round scalars decided by thread 0 (FP64 arithmetic once per CTA, not per thread):
    // status (-1: go on), inner scale 1 / ||r|| (FP32), inner threshold^2, the FP64 scale split
    // into hi + lo floats, the inner iteration cap
    __shared__ int s_status, s_icap;
    __shared__ float s_inv, s_target2, s_sh, s_sl;
    // the system's FP64 norms and refinement count, kept by thread 0 (no registers in the others)
    __shared__ double s_bn, s_rn, s_prev;
    __shared__ int s_ref;
    static_assert(RTPB == 1024, "one partial per lane in the final warp sums");
    for (int k = tid; k < md.rbeg[md.ns]; k += RTPB) sdesc[k] = md.rdesc[k];
    auto all_sum3 = [&](float (*buf)[3], float a0, float a1, float a2) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
            buf[wid][0] = a0;
            buf[wid][1] = a1;
            buf[wid][2] = a2;
        }
        __syncthreads();
        float3 t = make_float3(buf[lane][0], buf[lane][1], buf[lane][2]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
            t.z += __shfl_xor_sync(0xffffffffu, t.z, o);
        }
        return t;
    };
    // mixed-radix digits (d, n_0 .. n_{M-1}) of this thread's first element and of the stride RTPB
    int d0, n0[MAXM], inc[MAXM], incd;
    d0 = (int)fdiv((unsigned)tid, md.fd_nnu);
    decode<M>(md, tid - d0 * md.Nnu, n0);
    incd = (int)fdiv((unsigned)RTPB, md.fd_nnu);
    decode<M>(md, RTPB - incd * md.Nnu, inc);
    auto advance = [&](int& d, int (&n)[MAXM]) {
        int c = 0;
#pragma unroll
        for (int m = M - 1; m >= 0; --m) {
            const int v = n[m] + inc[m] + c;
            c = v >= md.nb[m];
            n[m] = c ? v - md.nb[m] : v;
        }
        d += incd + c;
    };
    // quad digits (d, n_0 .. n_{M-3}, b, n_{M-1}), radices (n_s, nb_0 .. nb_{M-3}, nb_{M-2} / 4,
    // nb_{M-1}): those of this thread's first quad (u = tid), then steps of RTPB quads
    const int S = md.nb[M - 1], NQ = N >> 2;
    const int S8 = S * (int)sizeof(float2);
    auto qstart = [&](int& d, int (&n)[MAXM]) {
        unsigned rem = (unsigned)tid;
#pragma unroll
        for (int m = M - 1; m >= 0; --m) {
            const unsigned q = fdiv(rem, a.qfd[m]);
            n[m] = (int)(rem - q * (unsigned)a.qfd[m].d);
            rem = q;
        }
#pragma unroll
        for (int m = M; m < MAXM; ++m) n[m] = 0;
        d = (int)rem;
    };
    auto qadvance = [&](int& d, int (&n)[MAXM]) {
        int c = 0;
#pragma unroll
        for (int m = M - 1; m >= 0; --m) {
            const int v = n[m] + a.qinc[m] + c;
            c = v >= a.qfd[m].d;
            n[m] = c ? v - a.qfd[m].d : v;
        }
        d += a.qincd + c;
    };
    for (;;) {
        __syncthreads();  // the previous system's shared data is no longer read
        for (int w = tid; w < NW; w += RTPB) bmask[w] = 0u;
        if (tid == 0) {
            const int q = atomicAdd(a.counter, 1);
            snext = q < a.nsys ? a.nsys - 1 - q : -1;
            s_bn = s_rn = s_prev = 0.0;
            s_ref = 0;
        }
        __syncthreads();
        const int s = snext;
        if (s < 0) break;
        const long long so = (long long)s * N;
        const int e = a.sys_e[s];
        const float2* dg = a.diag32 + (long long)e * N;
        const float2* di = dinv + (long long)e * N;
        const float4* dgdf = a.diagdf + (long long)e * N;
        float4* xs = a.xs + so;
        float2* x = xw + so;
        float2* r = rw + so;
        int iters = 0, status = -1;
        float inres = 1.f;
        // the split solution: written to xs by the first x update (never read before it: no zero
        // fill needed) and to XS in shared memory by every x update, where the next residual
        // reads it; xs_smem: XS holds it (not yet overwritten by an inner solve's p and q)
        bool xs_set = false, xs_smem = false;
        for (int k = 0;; ++k) {
            // ---- r = b - A x in double-float (x = 0 in the first round); its FP32 hi part to r
            if (k > 0) {
                for (int i = tid; i < H; i += RTPB) XS[-1 - i] = XS[N + i] = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int i = tid; i < md.nrct; i += RTPB) rows[i] = md.rctd[i];
                __syncthreads();
            }
            float nrm = 0.f;
            {
                int d = d0, n[MAXM];
#pragma unroll
                for (int m = 0; m < MAXM; ++m) n[m] = n0[m];
                float4 gn = k > 0 && tid < N ? dgdf[tid] : make_float4(0.f, 0.f, 0.f, 0.f);
                for (int i = tid; i < N; i += RTPB) {
                    if (i != tid) advance(d, n);
                    const float4 g = gn;  // the diagonal of this element; the next one's load issued now
                    if (k > 0 && i + RTPB < N) gn = dgdf[i + RTPB];
                    // the (re, im) pair as one packed double-float accumulator (hi parts, lo parts)
                    float2 sh = make_float2(0.f, 0.f), sl = make_float2(0.f, 0.f);
                    if (k == 0 || ((bmask[i >> 5] >> (i & 31)) & 1u)) {
                        const double2 bb = a.b64[so + i];
                        if ((__double_as_longlong(bb.x) | __double_as_longlong(bb.y)) != 0) {
                            sh = make_float2((float)bb.x, (float)bb.y);
                            sl = make_float2((float)(bb.x - (double)sh.x), (float)(bb.y - (double)sh.y));
                            if (k == 0) atomicOr(&bmask[i >> 5], 1u << (i & 31));
                        }
                    }
                    if (k > 0) {
                        // - diag x: (re, im) += (-g_re)(x_re, x_im) + (g_im, -g_im)(x_im, x_re)
                        const float4 xv = XS[i];
                        df_fma2(sh, sl, make_float2(-g.x, -g.x), make_float2(-g.z, -g.z), make_float2(g.x, g.x),
                                make_float2(xv.x, xv.y), make_float2(xv.z, xv.w));
                        df_fma2(sh, sl, make_float2(g.y, -g.y), make_float2(g.w, -g.w), make_float2(-g.y, g.y),
                                make_float2(xv.y, xv.x), make_float2(xv.w, xv.z));
                        int kk = md.rbeg[d];
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const int kend = kk + md.rcnt[d][m];
                            const float2* row = rows + n[m];
#pragma unroll 4
                            for (; kk < kend; ++kk) {
                                const int4 q = sdesc[kk];
                                float2 c = row[q.x >> 3];
                                if constexpr (SEC) {
                                    if (q.z >= 0) {  // a second mode's factor t (FP64 table, split hi + lo)
                                        const double tv = md.tab64[q.z + nsel<M>(n, q.w)];
                                        const float th = (float)tv, tl = (float)(tv - (double)th);
                                        const float ph = c.x * th;
                                        c = make_float2(ph, fmaf(c.x, th, -ph) + fmaf(c.x, tl, c.y * th));
                                    }
                                }
                                const float4 v = XS[i + (q.y >> 3)];  // neighbours outside [0, N) read the zero halo
                                df_fma2(sh, sl, make_float2(c.x, c.x), make_float2(c.y, c.y), make_float2(-c.x, -c.x),
                                        make_float2(v.x, v.y), make_float2(v.z, v.w));
                            }
                        }
                    }
                    const float2 hi = fadd2(sh, sl);  // the FP32 part of the renormalised pair
                    r[i] = hi;
                    nrm = fmaf(hi.x, hi.x, fmaf(hi.y, hi.y, nrm));
                }
            }
            // ||r||^2: FP32 within a warp, FP64 across warps (warp 0); the refinement checks in
            // thread 0, the outcome broadcast through shared memory
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
            if (lane == 0) redD[wid] = (double)nrm;
            __syncthreads();
            if (wid == 0) {
                double t = redD[lane];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                if (lane == 0) {
                    int st_ = -1;
                    s_rn = sqrt(t);
                    if (k == 0) {
                        s_bn = a.bn2 ? sqrt(a.bn2[s]) : s_rn;
                        if (s_bn == 0.0) {
                            st_ = VBK_SYS_ZERO_RHS;
                            s_rn = 0.0;
                        }
                    } else {
                        s_ref += 1;
                    }
                    if (st_ < 0) {
                        if (!isfinite(s_rn)) st_ = VBK_SYS_NAN;
                        else if (s_rn <= a.tol * s_bn) st_ = VBK_SYS_CONVERGED;
                        else if (a.stall_check && k > 0 && !(s_rn <= 0.9 * s_prev)) st_ = VBK_SYS_STALLED;  // FP32 inner solve no longer helps
                        else if (s_ref >= a.max_refine || iters >= a.max_iter) st_ = VBK_SYS_MAX_ITER;
                    }
                    s_status = st_;
                    if (st_ < 0) {
                        s_prev = s_rn;
                        s_inv = (float)(1.0 / s_rn);
                        const float tg = (float)fmax(a.inner_tol, 0.3 * a.tol * s_bn / s_rn);
                        s_target2 = tg * tg;
                        s_sh = (float)s_rn;
                        s_sl = (float)(s_rn - (double)s_sh);
                        s_icap = a.inner_cap > 0 ? (int)min((long long)a.max_iter, (long long)iters + a.inner_cap) : a.max_iter;
                    }
                }
            }
            __syncthreads();
            if (s_status >= 0) {
                status = s_status;
                break;
            }
            const float inv = s_inv, target2 = s_target2;
            const int icap = s_icap;
            // ---- inner FP32 COCG on r / ||r|| (x = 0, z = B^-1 r, p = z, rho = r^T z)
            xs_smem = false;
            for (int i = tid; i < md.nrct; i += RTPB) rows[i] = md.rct[i];
            for (int i = tid; i < H; i += RTPB) P[-1 - i] = P[N + i] = make_float2(0.f, 0.f);
            __syncthreads();  // XS (which overlays P) fully read
            float2 rho, beta = make_float2(0.f, 0.f);
            {
                float rz_x = 0.f, rz_y = 0.f;
                for (int i = tid; i < N; i += RTPB) {
                    const float2 rv = r[i];
                    const float2 rn2 = make_float2(rv.x * inv, rv.y * inv);
                    r[i] = rn2;
                    const float2 zi = a.pmode == 0 ? cmul<float>(rn2, di[i]) : rn2;
                    P[i] = zi;
                    rz_x += rn2.x * zi.x - rn2.y * zi.y;
                    rz_y += rn2.x * zi.y + rn2.y * zi.x;
                }
                const float3 t = all_sum3(redB, 0.f, rz_x, rz_y);
                rho = make_float2(t.y, t.z);
            }
            bool wrote_x = false;
            float rr = 0.f;
            const int budget = max(0, icap - iters);
            for (int it = 0; it < budget; ++it) {
                float pq_x = 0.f, pq_y = 0.f;
                if constexpr (QD) {
                    // quads: q = diag p - sum_points c p[nu + delta] for four elements per step
                    int d, n[MAXM];
                    qstart(d, n);
                    for (int u = tid; u < NQ; u += RTPB) {
                        if (u != tid) qadvance(d, n);
                        const int w = (int)fdiv((unsigned)u, md.fd_nb[M - 1]);
                        const int i0 = 4 * S * w + (u - w * S);
                        float2 acc[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[c] = make_float2(0.f, 0.f);
                        const char* Pq = reinterpret_cast<const char*>(P + i0);
                        int kk = md.rbeg[d];
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const int kend = kk + md.rcnt[d][m];
                            if (m == M - 2) {  // four consecutive (-c, -c) pairs, two float4 loads
                                const char* row = reinterpret_cast<const char*>(rows) + n[m] * 32;
#pragma unroll 1
                                for (; kk < kend; ++kk) {
                                    const int4 q = sdesc[kk];
                                    const float4 c01 = *reinterpret_cast<const float4*>(row + q.x);
                                    const float4 c23 = *reinterpret_cast<const float4*>(row + q.x + 16);
                                    const char* ap = Pq + q.y;  // zero halo outside [0, N)
                                    acc[0] = ffma2(make_float2(c01.x, c01.y), *reinterpret_cast<const float2*>(ap), acc[0]);
                                    acc[1] = ffma2(make_float2(c01.z, c01.w), *reinterpret_cast<const float2*>(ap + S8), acc[1]);
                                    acc[2] = ffma2(make_float2(c23.x, c23.y), *reinterpret_cast<const float2*>(ap + 2 * S8), acc[2]);
                                    acc[3] = ffma2(make_float2(c23.z, c23.w), *reinterpret_cast<const float2*>(ap + 3 * S8), acc[3]);
                                }
                            } else {  // one (-c, -c) pair for the four
                                const char* row = reinterpret_cast<const char*>(rows) + n[m] * 8;
#pragma unroll 1
                                for (; kk < kend; ++kk) {
                                    const int4 q = sdesc[kk];
                                    const float2 cc = *reinterpret_cast<const float2*>(row + q.x);
                                    const char* ap = Pq + q.y;
#pragma unroll
                                    for (int c = 0; c < 4; ++c)
                                        acc[c] = ffma2(cc, *reinterpret_cast<const float2*>(ap + c * S8), acc[c]);
                                }
                            }
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float2 pi = P[i0 + c * S], g = dg[i0 + c * S];
                            const float2 v = make_float2(acc[c].x + g.x * pi.x - g.y * pi.y,
                                                         acc[c].y + g.x * pi.y + g.y * pi.x);
                            Q[i0 + c * S] = v;
                            pq_x += pi.x * v.x - pi.y * v.y;
                            pq_y += pi.x * v.y + pi.y * v.x;
                        }
                    }
                } else {
                    int d = d0, n[MAXM];
#pragma unroll
                    for (int m = 0; m < MAXM; ++m) n[m] = n0[m];
                    // the diagonal of RC consecutive elements of this thread is loaded ahead (L2 latency)
                    constexpr int RC = 4;
                    for (int i0 = tid; i0 < N; i0 += RC * RTPB) {
                        float2 dgv[RC];
#pragma unroll
                        for (int c = 0; c < RC; ++c) {
                            const int ic = i0 + c * RTPB;
                            dgv[c] = ic < N ? dg[ic] : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int c = 0; c < RC; ++c) {
                        const int i = i0 + c * RTPB;
                        if (i >= N) break;
                        if (i != tid) advance(d, n);
                        const float2 pi = P[i];
                        float2 acc = cmul<float>(dgv[c], pi);
                        const char* Pi = reinterpret_cast<const char*>(P + i);
                        int kk = md.rbeg[d];
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const int kend = kk + md.rcnt[d][m];
                            const char* row = reinterpret_cast<const char*>(rows) + n[m] * 8;
#pragma unroll 4
                            for (; kk < kend; ++kk) {
                                const int4 q = sdesc[kk];
                                float2 cc = *reinterpret_cast<const float2*>(row + q.x);  // (-c, -c)
                                if constexpr (SEC) {
                                    if (q.z >= 0) {
                                        const float t = md.tab32[q.z + nsel<M>(n, q.w)];
                                        cc.x *= t;
                                        cc.y *= t;
                                    }
                                }
                                acc = ffma2(cc, *reinterpret_cast<const float2*>(Pi + q.y), acc);  // zero halo outside
                            }
                        }
                        Q[i] = acc;
                        pq_x += pi.x * acc.x - pi.y * acc.y;
                        pq_y += pi.x * acc.y + pi.y * acc.x;
                        }
                    }
                }
                const float3 pq = all_sum3(redA, pq_x, pq_y, 0.f);
                const float den = pq.x * pq.x + pq.y * pq.y;
                if (!(den > 0.f) || !isfinite(den)) {
                    status = isfinite(den) ? VBK_SYS_BREAKDOWN : VBK_SYS_NAN;
                    break;
                }
                const float2 al = make_float2((rho.x * pq.x + rho.y * pq.y) / den, (rho.y * pq.x - rho.x * pq.y) / den);
                float rr_l = 0.f, rz_x = 0.f, rz_y = 0.f;
                // x, r and 1/diag of UC elements of this thread are loaded ahead (L2 latency)
                constexpr int UC = 2;
                for (int i0 = tid; i0 < N; i0 += UC * RTPB) {
                    float2 xl[UC], rl[UC], dl[UC];
#pragma unroll
                    for (int c = 0; c < UC; ++c) {
                        const int ic = i0 + c * RTPB;
                        const bool ok = ic < N;
                        xl[c] = ok && it > 0 ? x[ic] : make_float2(0.f, 0.f);
                        rl[c] = ok ? r[ic] : make_float2(0.f, 0.f);
                        dl[c] = ok && a.pmode == 0 ? di[ic] : make_float2(1.f, 0.f);
                    }
#pragma unroll
                    for (int c = 0; c < UC; ++c) {
                        const int i = i0 + c * RTPB;
                        if (i >= N) break;
                        const float2 pi = P[i], qi = Q[i];
                        float2 xv = xl[c];
                        xv.x += al.x * pi.x - al.y * pi.y;
                        xv.y += al.x * pi.y + al.y * pi.x;
                        x[i] = xv;
                        float2 rv = rl[c];
                        rv.x -= al.x * qi.x - al.y * qi.y;
                        rv.y -= al.x * qi.y + al.y * qi.x;
                        r[i] = rv;
                        const float2 zi = a.pmode == 0 ? cmul<float>(rv, dl[c]) : rv;
                        Q[i] = zi;
                        rr_l += rv.x * rv.x + rv.y * rv.y;
                        rz_x += rv.x * zi.x - rv.y * zi.y;
                        rz_y += rv.x * zi.y + rv.y * zi.x;
                    }
                }
                const float3 sums = all_sum3(redB, rr_l, rz_x, rz_y);
                wrote_x = true;
                iters += 1;
                rr = sums.x;
                if (!isfinite(sums.x) || !isfinite(sums.y) || !isfinite(sums.z) || sums.x <= target2 || iters >= icap) break;
                const float rden = rho.x * rho.x + rho.y * rho.y;
                if (!(sums.y * sums.y + sums.z * sums.z > 0.f) || !(rden > 0.f)) {
                    status = VBK_SYS_BREAKDOWN;
                    break;
                }
                beta = make_float2((sums.y * rho.x + sums.z * rho.y) / rden, (sums.z * rho.x - sums.y * rho.y) / rden);
                rho = make_float2(sums.y, sums.z);
                for (int i = tid; i < N; i += RTPB) {
                    const float2 pi = P[i], zi = Q[i];
                    P[i] = make_float2(zi.x + beta.x * pi.x - beta.y * pi.y, zi.y + beta.x * pi.y + beta.y * pi.x);
                }
                __syncthreads();
            }
            inres = sqrtf(rr);
            // ---- x += scale d in double-float (each thread its own elements)
            if (wrote_x) {  // P and Q are dead: XS (over them) receives the new solution as well
                const float sh = s_sh, sl = s_sl;
                for (int i = tid; i < N; i += RTPB) {
                    const float2 dv = x[i];
                    float4 X = xs_set ? xs[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                    df_fma(X.x, X.z, sh, sl, dv.x, 0.f);
                    df_fma(X.y, X.w, sh, sl, dv.y, 0.f);
                    const float2 re = df_norm(X.x, X.z), im = df_norm(X.y, X.w);
                    X = make_float4(re.x, im.x, re.y, im.y);
                    xs[i] = X;
                    XS[i] = X;
                }
                xs_set = true;
            } else {  // no new solution, but the inner solve wrote over XS: restore it
                for (int i = tid; i < N; i += RTPB) XS[i] = xs_set ? xs[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            xs_smem = true;
            if (status >= 0) break;
            __syncthreads();  // P, Q fully read before the next residual stages XS over them
        }
        // ---- psi = hi + lo in FP64 (from XS after a final residual, else from xs; zero if no
        // solution was ever formed), and the system's record
        double2* psi = a.psi + so;
        if (!xs_smem) {
            __syncthreads();  // an inner solve may still be reading P / Q over XS
            for (int i = tid; i < N; i += RTPB) XS[i] = xs_set ? xs[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
        }
        for (int i = tid; i < N; i += RTPB) {
            const float4 v = XS[i];
            psi[i] = make_double2(f2d_exact(v.x) + f2d_exact(v.z), f2d_exact(v.y) + f2d_exact(v.w));
        }
        if (tid == 0) {
            SysState& S = a.st[s];
            S.status = status < 0 ? VBK_SYS_MAX_ITER : status;
            S.iters = iters;
            S.refines = s_ref;
            S.rnorm = s_rn;
            S.bnorm = s_bn;
            S.inres = (double)inres;
        }
    }
}
inline bool resident_ok(const DevModel& md);
inline size_t solve_resident_smem(const DevModel& md) {
    const size_t pq = (size_t)(2 * md.N + 2 * md.rhalo) * 8, xsb = (size_t)(md.N + 2 * md.rhalo) * 16;
    return std::max(pq, xsb) + (((size_t)md.nrct * 8 + 15) & ~(size_t)15) + (size_t)((md.N + 31) / 32) * 4 + 16;
}
// the instance for a model: a second mode's factor per point (SEC), else quads when n_{M-2} runs
// over a multiple of 4 functions, else one element per step
using SolveResidentFn = void (*)(DevModel, ClArgs, float2*, float2*, const float2*);
template <int M> SolveResidentFn solve_resident_fn(const DevModel& md) {
    if (md.rsec) return k_solve_resident<M, true, false>;
    if constexpr (M >= 2) {
        if (md.nb[M - 2] % 4 == 0) return k_solve_resident<M, false, true>;
    }
    return k_solve_resident<M, false, false>;
}
// the quad digit radices and the digits of the stride RTPB (quad loops of k_solve_resident)
inline void set_quad_args(const DevModel& md, int M, ClArgs& a) {
    for (int m = 0; m < MAXM; ++m) {
        a.qfd[m] = make_fastdiv(1);
        a.qinc[m] = 0;
    }
    a.qincd = 0;
    if (M < 2 || md.nb[M - 2] % 4 != 0) return;
    int rem = RTPB;
    for (int m = M - 1; m >= 0; --m) {
        const int rad = m == M - 2 ? md.nb[m] / 4 : md.nb[m];
        a.qfd[m] = make_fastdiv(rad);
        a.qinc[m] = rem % rad;
        rem /= rad;
    }
    a.qincd = rem;
}
template <int M> bool prepare_solve_resident(const DevModel& md) {
    if (!resident_ok(md) || solve_resident_smem(md) > 220 * 1024) return false;
    const cudaError_t ce = cudaFuncSetAttribute(solve_resident_fn<M>(md), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)solve_resident_smem(md));
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

template <int M> bool prepare_residual_res(const DevModel& md) {
    if (md.rsec || residual_res_smem(md) > 220 * 1024) return false;
    if (cudaFuncSetAttribute(k_residual_res<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)residual_res_smem(md)) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// y = A x (or b - A x) in FP32 for S systems per CTA (grid: groups of S list entries): each
// system's x is staged once in shared memory with a zero halo (every x entry leaves L2/HBM once,
// neighbours come from shared memory), coefficients from the primary-mode rows as in the
// resident COCG kernel, shared by the S systems.  One partial per system: x^T y (red = 1) or
// ||y||^2 (red = 2) in part[s].
template <int M, int S>
__global__ void __launch_bounds__(RTPB, 1) k_matvec_sys(DevModel md, const int* __restrict__ sys_e, Sel sel, int nlist,
                                                       const float2* __restrict__ diag, const float2* __restrict__ x,
                                                       long long xs, float2* __restrict__ y, long long ys,
                                                       const double2* __restrict__ b, double2* __restrict__ part, int red) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = md.N, H = md.rhalo, NH = N + 2 * H;
    float2* Xb = reinterpret_cast<float2*>(smraw) + H;  // system t: Xb + t * NH
    float2* sct = reinterpret_cast<float2*>(smraw) + S * NH;
    __shared__ int4 sdesc[MAXS * 64];
    __shared__ float2 redsh[RTPB / 32];
    const int tid = threadIdx.x;
    int sy[S];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        const int li = blockIdx.x * S + t;
        int s = -1;
        if (li < nlist) {
            s = sel.list ? sel.list[li] : li;
            if (s >= 0 && sel.act && !sel.act[s]) s = -1;
        }
        sy[t] = s;
    }
    for (int k = tid; k < md.nrct; k += RTPB) sct[k] = md.rct[k];
    for (int k = tid; k < md.rbeg[md.ns]; k += RTPB) sdesc[k] = md.rdesc[k];
#pragma unroll
    for (int t = 0; t < S; ++t) {
        float2* X = Xb + t * NH;
        for (int k = tid; k < H; k += RTPB) X[-1 - k] = X[N + k] = make_float2(0.f, 0.f);
        const float2* xv = x + (long long)(sy[t] < 0 ? 0 : sy[t]) * xs;
        for (int i = tid; i < N; i += RTPB) X[i] = sy[t] < 0 ? make_float2(0.f, 0.f) : xv[i];
    }
    __syncthreads();
    float2 loc[S];
#pragma unroll
    for (int t = 0; t < S; ++t) loc[t] = make_float2(0.f, 0.f);
    for (int i = tid; i < N; i += RTPB) {
        const int d = (int)fdiv((unsigned)i, md.fd_nnu), nu = i - d * md.Nnu;
        int n[MAXM];
        decode<M>(md, nu, n);
        float2 acc[S], xi[S];
#pragma unroll
        for (int t = 0; t < S; ++t) {
            xi[t] = Xb[t * NH + i];
            acc[t] = sy[t] < 0 ? make_float2(0.f, 0.f) : cmul<float>(diag[(long long)sys_e[sy[t]] * N + i], xi[t]);
        }
        const char* Xi = reinterpret_cast<const char*>(Xb + i);
        int k = md.rbeg[d];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int kend = k + md.rcnt[d][m];
            const char* row = reinterpret_cast<const char*>(sct) + n[m] * 8;
#pragma unroll 4
            for (; k < kend; ++k) {
                const int4 q = sdesc[k];
                float2 cc = *reinterpret_cast<const float2*>(row + q.x);  // (-c, -c)
                if (q.z >= 0) {
                    const float tt = md.tab32[q.z + nsel<M>(n, q.w)];
                    cc.x *= tt;
                    cc.y *= tt;
                }
#pragma unroll
                for (int t = 0; t < S; ++t)  // neighbours outside [0, N) read the zero halo
                    acc[t] = ffma2(cc, *reinterpret_cast<const float2*>(Xi + (size_t)t * NH * 8 + q.y), acc[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < S; ++t) {
            if (sy[t] < 0) continue;
            float2 out = acc[t];
            if (b) {
                const double2 bb = b[(long long)sy[t] * N + i];
                out = make_float2((float)bb.x - out.x, (float)bb.y - out.y);
            }
            y[(long long)sy[t] * ys + i] = out;
            if (red == 1) loc[t] = cfma<float>(xi[t], out, loc[t]);
            else if (red == 2) loc[t].x = fmaf(out.x, out.x, fmaf(out.y, out.y, loc[t].x));
        }
    }
    if (red) {
#pragma unroll
        for (int t = 0; t < S; ++t) {
            const double2 tot = block_sum_c<float>(loc[t], redsh);
            if (tid == 0 && sy[t] >= 0) part[sy[t]] = tot;
        }
    }
}
inline size_t matvec_sys_smem(const DevModel& md, int S) {
    return (size_t)(S * (md.N + 2 * md.rhalo) + md.nrct) * sizeof(float2) + 16;
}

// shared memory of the resident kernel: p (with its halo), q, the oscillator tables and the
// primary-mode coefficient rows (FP32)
inline size_t resident_smem(const DevModel& md) {
    return (size_t)(2 * md.N + 2 * md.rhalo + md.nrct) * sizeof(float2) + 16;
}
inline bool resident_ok(const DevModel& md) {
    if (!md.rok || resident_smem(md) > 220 * 1024) return false;
    for (int d = 0; d < md.ns; ++d)
        if (md.ebeg[d + 1] - md.ebeg[d] > 64) return false;
    return true;
}
template <int M> int prepare_resident(const DevModel& md) {
    const cudaError_t ce =
        md.rsec ? cudaFuncSetAttribute(k_cocg_resident<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)resident_smem(md))
                : cudaFuncSetAttribute(k_cocg_resident<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)resident_smem(md));
    return ce == cudaSuccess ? VBK_OK : vbk_cuda_fail(ce, "resident COCG shared-memory opt-in");
}

// ---------------------------------------------------------------------------- GMRES
// Restarted GMRES(m) with right preconditioning (Sec. III.A; Saad & Schultz): Arnoldi
// A B^-1 V_n = V_{n+1} H_n with classical Gram-Schmidt applied twice (CGS2), the
// (n+1) x n least-squares problem solved by complex Givens rotations in FP64.
// V of system s: [s][k = 0..m][N] in the inner precision.

// partial h_k = sum_i conj(V_k[i]) w[i], k = 0..j;  part[s][blk][k], (m+1) slots
template <class R>
__global__ void __launch_bounds__(TPB) k_vdots(int N, int m, Sel sel, const cx<R>* __restrict__ V,
                                              int j, const cx<R>* __restrict__ w, double2* __restrict__ part) {
    __shared__ double2 sh[(TPB / 32) * 257];
    const int s = sel_sys(sel);
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const long long vs = (long long)(m + 1) * N;
    const cx<R>* Vs = V + s * vs;
    const cx<R>* ws = w + (long long)s * N;
    const int i0 = blockIdx.x * VCHUNK + threadIdx.x;
    cx<R> wl[VEPT];
#pragma unroll
    for (int u = 0; u < VEPT; ++u) {
        const int i = i0 + u * TPB;
        wl[u] = i < N ? ws[i] : mkc<R>(0, 0);
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int k = 0; k <= j; ++k) {
        const cx<R>* vk = Vs + (long long)k * N;
        cx<R> a = mkc<R>(0, 0);
#pragma unroll
        for (int u = 0; u < VEPT; ++u) {
            const int i = i0 + u * TPB;
            if (i < N) {
                const cx<R> t = cconjmul<R>(vk[i], wl[u]);
                a.x += t.x;
                a.y += t.y;
            }
        }
        const cx<R> dv = warp_sum_c<R>(a);
        if (lane == 0) sh[wp * 257 + k] = cvt_to_d<R>(dv);
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= j; k += blockDim.x) {
        double2 t = make_double2(0.0, 0.0);
        for (int q = 0; q < TPB / 32; ++q) {
            t.x += sh[q * 257 + k].x;
            t.y += sh[q * 257 + k].y;
        }
        part[((long long)s * gridDim.x + blockIdx.x) * (m + 1) + k] = t;
    }
}

// h[s][k] = sum over blocks of part[s][blk][k]
// h[s][k] = sum over the nb per-block partials of dot k (k = 0 .. j) of system s.  Grid:
// (dot groups of HR_K, systems); thread (x, y) sums the partials b = y, y + HR_G, .. of dot
// k0 + x (consecutive dots: coalesced rows of partials), two accumulators in flight, then the
// HR_G sums of a dot are added in shared memory.
constexpr int HR_K = 32, HR_G = 8;
__global__ void __launch_bounds__(HR_K * HR_G) k_hreduce(int nsys, int m, const int* __restrict__ act, int j,
                                                       const double2* __restrict__ part, int nb, double2* __restrict__ h) {
    __shared__ double2 sh[HR_G][HR_K];
    const int s = blockIdx.y;
    if (s >= nsys || !act[s]) return;
    const int k = blockIdx.x * HR_K + threadIdx.x;
    double2 t0 = make_double2(0.0, 0.0), t1 = t0;
    if (k <= j) {
        const double2* pk = part + (long long)s * nb * (m + 1) + k;
        int b = threadIdx.y;
        for (; b + HR_G < nb; b += 2 * HR_G) {
            const double2 v0 = pk[(long long)b * (m + 1)], v1 = pk[(long long)(b + HR_G) * (m + 1)];
            t0.x += v0.x;
            t0.y += v0.y;
            t1.x += v1.x;
            t1.y += v1.y;
        }
        if (b < nb) {
            const double2 v0 = pk[(long long)b * (m + 1)];
            t0.x += v0.x;
            t0.y += v0.y;
        }
    }
    sh[threadIdx.y][threadIdx.x] = make_double2(t0.x + t1.x, t0.y + t1.y);
    __syncthreads();
    if (threadIdx.y == 0 && k <= j) {
        double2 t = sh[0][threadIdx.x];
#pragma unroll
        for (int q = 1; q < HR_G; ++q) {
            t.x += sh[q][threadIdx.x].x;
            t.y += sh[q][threadIdx.x].y;
        }
        h[(long long)s * (m + 1) + k] = t;
    }
}

// w -= sum_k V_k h_k; then (mode 0) partial dots conj(V_k) w, or (mode 1) partial ||w||^2
template <class R>
__global__ void __launch_bounds__(TPB) k_vupdate(int N, int m, Sel sel, const cx<R>* __restrict__ V,
                                                int j, const double2* __restrict__ h, cx<R>* __restrict__ w, int mode,
                                                double2* __restrict__ part) {
    __shared__ double2 sh[(TPB / 32) * 257];
    __shared__ cx<R> hs[257];
    const int s = sel_sys(sel);
    if (s < 0 || (sel.act && !sel.act[s])) return;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) hs[k] = cvt_from_d<R>(h[(long long)s * (m + 1) + k]);
    __syncthreads();
    const long long vs = (long long)(m + 1) * N;
    const cx<R>* Vs = V + s * vs;
    cx<R>* ws = w + (long long)s * N;
    const int i0 = blockIdx.x * VCHUNK + threadIdx.x;
    cx<R> wl[VEPT];
#pragma unroll
    for (int u = 0; u < VEPT; ++u) {
        const int i = i0 + u * TPB;
        wl[u] = i < N ? ws[i] : mkc<R>(0, 0);
    }
    for (int k = 0; k <= j; ++k) {
        const cx<R>* vk = Vs + (long long)k * N;
        const cx<R> hk = hs[k];
#pragma unroll
        for (int u = 0; u < VEPT; ++u) {
            const int i = i0 + u * TPB;
            if (i < N) wl[u] = csub<R>(wl[u], cmul<R>(vk[i], hk));
        }
    }
#pragma unroll
    for (int u = 0; u < VEPT; ++u) {
        const int i = i0 + u * TPB;
        if (i < N) ws[i] = wl[u];
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (mode == 0) {
        for (int k = 0; k <= j; ++k) {
            const cx<R>* vk = Vs + (long long)k * N;
            cx<R> a = mkc<R>(0, 0);
#pragma unroll
            for (int u = 0; u < VEPT; ++u) {
                const int i = i0 + u * TPB;
                if (i < N) {
                    const cx<R> t = cconjmul<R>(vk[i], wl[u]);
                    a.x += t.x;
                    a.y += t.y;
                }
            }
            const cx<R> dv = warp_sum_c<R>(a);
            if (lane == 0) sh[wp * 257 + k] = cvt_to_d<R>(dv);
        }
        __syncthreads();
        for (int k = threadIdx.x; k <= j; k += blockDim.x) {
            double2 t = make_double2(0.0, 0.0);
            for (int q = 0; q < TPB / 32; ++q) {
                t.x += sh[q * 257 + k].x;
                t.y += sh[q * 257 + k].y;
            }
            part[((long long)s * gridDim.x + blockIdx.x) * (m + 1) + k] = t;
        }
    } else {
        R a = 0;
#pragma unroll
        for (int u = 0; u < VEPT; ++u) a += cabs2<R>(wl[u]);
        const double2 tot = block_sum_c<R>(mkc<R>(a, 0), reinterpret_cast<cx<R>*>(sh));
        if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = tot;
    }
}

// Column j of the Hessenberg matrix, Givens rotations and the residual estimate (FP64).
// Givens QR step of every active system, one warp per system (GV_W systems per block): the
// lanes sum the norm partials and stage the new Hessenberg column h1 + h2 and the j earlier
// rotations in shared memory; lane 0 then applies the rotations with the running entry in
// registers (no global load inside the dependent chain) and forms the new rotation.
constexpr int GV_W = 4;
constexpr int GV_MAXM = 256;  // the restart length is at most 256
__global__ void __launch_bounds__(32 * GV_W) k_givens(int nsys, int m, SysState* __restrict__ st, int* __restrict__ act,
                         const double2* __restrict__ h1, const double2* __restrict__ h2,
                         const double2* __restrict__ part_n, int nb, double2* __restrict__ H, double* __restrict__ cs,
                         double2* __restrict__ sn, double2* __restrict__ g, double* __restrict__ inv_h, int max_iter,
                         int* __restrict__ count, int* __restrict__ ilist) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * GV_W + (threadIdx.x >> 5);
    if (s >= nsys || !act[s]) return;
    SysState& S = st[s];
    const int j = S.j;
    double rr = 0.0;
    __shared__ double scs[GV_W][GV_MAXM];
    __shared__ double2 ssn[GV_W][GV_MAXM], scol[GV_W][GV_MAXM + 1];
    const int wv = threadIdx.x >> 5;
    for (int k = lane; k < nb; k += 32) rr += part_n[(long long)s * nb + k].x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
    double* csv = cs + (long long)s * m;
    double2* snv = sn + (long long)s * m;
    const double2* h1s = h1 + (long long)s * (m + 1);
    const double2* h2s = h2 + (long long)s * (m + 1);
    for (int k = lane; k < j; k += 32) {
        scs[wv][k] = csv[k];
        ssn[wv][k] = snv[k];
    }
    for (int k = lane; k <= j; k += 32) scol[wv][k] = make_double2(h1s[k].x + h2s[k].x, h1s[k].y + h2s[k].y);
    __syncwarp();
    if (lane != 0) return;
    const double hn = sqrt(rr);
    double2* Hc = H + ((long long)s * m + j) * (m + 1);  // column j
    // apply previous rotations to (h1 + h2)[0 .. j], hn; `cur` is the entry k of the column as
    // rotated by rotations 0 .. k-1
    double2* gv = g + (long long)s * (m + 1);
    double2 cur = scol[wv][0];
    for (int k = 0; k < j; ++k) {
        const double c = scs[wv][k];
        const double2 sk = ssn[wv][k];
        const double2 a = cur, b = scol[wv][k + 1];
        const double2 t1 = cmul<double>(sk, b);
        const double2 t2 = cconjmul<double>(sk, a);  // conj(s) a
        Hc[k] = make_double2(c * a.x + t1.x, c * a.y + t1.y);
        cur = make_double2(c * b.x - t2.x, c * b.y - t2.y);
    }
    // new rotation zeroing H[j+1][j]
    const double2 a = cur, b = make_double2(hn, 0.0);
    const double aa = sqrt(cabs2<double>(a)), bb = sqrt(cabs2<double>(b));
    double c;
    double2 sg;
    if (aa == 0.0) {
        c = 0.0;
        sg = make_double2(1.0, 0.0);
        Hc[j] = b;
    } else {
        const double nu = hypot(aa, bb);
        c = aa / nu;
        const double2 ph = make_double2(a.x / aa, a.y / aa);
        sg = cscale<double>(cmul<double>(ph, make_double2(b.x, -b.y)), 1.0 / nu);
        Hc[j] = cscale<double>(ph, nu);
    }
    Hc[j + 1] = make_double2(0.0, 0.0);
    csv[j] = c;
    snv[j] = sg;
    const double2 gj = gv[j];
    const double2 t = cconjmul<double>(sg, gj);
    gv[j + 1] = make_double2(-t.x, -t.y);
    gv[j] = cscale<double>(gj, c);
    S.j = j + 1;
    S.iters += 1;
    S.cycle_iters += 1;
    const double res = sqrt(cabs2<double>(gv[j + 1]));
    S.inres = res;
    inv_h[s] = hn > 0.0 ? 1.0 / hn : 0.0;
    if (!isfinite(res) || res <= S.target || hn == 0.0 || j + 1 >= m || S.iters >= max_iter) {
        act[s] = 0;
        return;
    }
    ilist[atomicAdd(count, 1)] = s;
}

template <class R>
__global__ void __launch_bounds__(TPB) k_vscale(int N, int m, Sel sel, const double* __restrict__ inv_h,
                                               const SysState* __restrict__ st, const cx<R>* __restrict__ w,
                                               cx<R>* __restrict__ V) {
    const int s = sel_sys(sel);
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const R inv = (R)inv_h[s];
    const int j = st[s].j;  // new basis vector index
    V[((long long)s * (m + 1) + j) * N + i] = cscale<R>(w[(long long)s * N + i], inv);
}

// y = H^-1 g (upper triangular, FP64) for the steps of the cycle; cyc[s] = 1 for systems
// that ran a cycle.
__global__ void k_tri_solve(int nsys, int m, const SysState* __restrict__ st, const int* __restrict__ cyc,
                            const double2* __restrict__ H, const double2* __restrict__ g, double2* __restrict__ y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || !cyc[s]) return;
    const int n = st[s].j;
    double2* ys = y + (long long)s * (m + 1);
    for (int k = n - 1; k >= 0; --k) {
        double2 acc = g[(long long)s * (m + 1) + k];
        for (int l = k + 1; l < n; ++l) acc = csub<double>(acc, cmul<double>(H[((long long)s * m + l) * (m + 1) + k], ys[l]));
        const double2 dk = H[((long long)s * m + k) * (m + 1) + k];
        ys[k] = (dk.x == 0.0 && dk.y == 0.0) ? make_double2(0.0, 0.0) : cdiv<double>(acc, dk);
    }
}

// u = sum_{k < j} y_k V_k (accumulated in the inner precision)
template <class R>
__global__ void __launch_bounds__(TPB) k_vcombine(int N, int m, Sel sel, const SysState* __restrict__ st,
                                                 const cx<R>* __restrict__ V, const double2* __restrict__ y,
                                                 cx<R>* __restrict__ u) {
    __shared__ cx<R> ys[257];
    const int s = sel_sys(sel);
    if (s < 0 || (sel.act && !sel.act[s])) return;
    const int n = st[s].j;
    for (int k = threadIdx.x; k < n; k += blockDim.x) ys[k] = cvt_from_d<R>(y[(long long)s * (m + 1) + k]);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const cx<R>* Vs = V + (long long)s * (m + 1) * N;
    cx<R> acc = mkc<R>(0, 0);
    for (int k = 0; k < n; ++k) acc = cfma<R>(ys[k], Vs[(long long)k * N + i], acc);
    u[(long long)s * N + i] = acc;
}

__global__ void k_gmres_cycle_start(int nsys, int m, const int* __restrict__ act, double2* __restrict__ g) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || !act[s]) return;
    g[(long long)s * (m + 1)] = make_double2(1.0, 0.0);  // ||inner rhs|| = 1 after scaling
}

// ------------------------------------------------------------------------------ driver
struct Runner {
    vbk_model* m;
    cudaStream_t st;
    bool timing;
    struct Pend {
        int id;
        cudaEvent_t a, b;
    };
    std::vector<Pend> pend;
    std::vector<cudaEvent_t> pool;
    int id(const char* name) {
        for (size_t k = 0; k < m->timers.size(); ++k)
            if (m->timers[k].name == name) return (int)k;
        KTimer t;
        t.name = name;
        m->timers.push_back(t);
        return (int)m->timers.size() - 1;
    }
    cudaEvent_t ev() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    template <typename K, typename... A>
    void go(const char* name, K kern, dim3 g, dim3 b, A... args) {
        go_smem(name, kern, g, b, 0, args...);
    }
    template <typename K, typename... A>
    void go_smem(const char* name, K kern, dim3 g, dim3 b, size_t smem, A... args) {
        if (g.x == 0 || g.y == 0) return;
        Pend pd{0, nullptr, nullptr};
        if (timing) {
            pd.id = id(name);
            pd.a = ev();
            pd.b = ev();
            cudaEventRecord(pd.a, st);
        }
        kern<<<g, b, smem, st>>>(args...);
        m->launches += 1;
        if (const cudaError_t ce = cudaPeekAtLastError(); ce != cudaSuccess) note_error(ce, name);
        if (timing) {
            cudaEventRecord(pd.b, st);
            m->timers[pd.id].launches += 1;
            pend.push_back(pd);
        }
    }
    // a launch made by `launch()` (returning its cudaError_t), timed like the others
    template <class F> void go_custom(const char* name, F launch) {
        Pend pd{0, nullptr, nullptr};
        if (timing) {
            pd.id = id(name);
            pd.a = ev();
            pd.b = ev();
            cudaEventRecord(pd.a, st);
        }
        const cudaError_t ce = launch();
        m->launches += 1;
        if (ce != cudaSuccess) note_error(ce, name);
        if (timing) {
            cudaEventRecord(pd.b, st);
            m->timers[pd.id].launches += 1;
            pend.push_back(pd);
        }
    }
    cudaError_t first_error = cudaSuccess;
    void note_error(cudaError_t e, const char* where) {
        if (first_error == cudaSuccess) {
            first_error = e;
            vbk_set_error(std::string("launch of ") + where + ": " + cudaGetErrorString(e));
        }
    }
    void flush() {  // call after a stream synchronisation
        for (auto& p : pend) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) m->timers[p.id].ms += ms;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pend.clear();
    }
    ~Runner() {
        for (auto& p : pend) {
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

template <class T> T* carve(char*& p, size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T* r = reinterpret_cast<T*>(p);
    p += bytes;
    return r;
}
template <class T> size_t carve_size(size_t count) { return (count * sizeof(T) + 255) & ~size_t(255); }

inline unsigned cdiv_u(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

struct DevPlanBuf {
    PlanDev pd{};
    void* mem = nullptr;
    bool staged = false;  // chains gathered through shared memory (k_block_staged)
    bool wide = false;    // p > PMAX: k_level_factor / k_level_apply
    int P = 0;            // register window of the staged kernel (>= p)
};

// Entries of the factor buffer of one energy: L * (p + 1) * nblk for the narrow kernels, the
// level blocks and the factorization window for the wide ones.
inline size_t factor_entries(const BlockPlan& bp, size_t N) {
    return bp.wide ? (size_t)level_factor_entries(bp.nblk, bp.K, bp.S) : N * (size_t)(bp.p + 1);
}

// Host tables of a block plan: element offset of every chain position, base element of
// every block, and (when the chain contains the fastest mode) its contiguous runs.
int upload_plan(const BlockPlan& bp, const vbk_model* m, cudaStream_t st, DevPlanBuf* out) {
    const int span = bp.span;
    std::vector<int> chain(bp.L), base(bp.nblk), run_off, run_c0;
    std::vector<int> nlast(bp.L, 0);
    for (int c = 0; c < bp.L; ++c) {
        int rem = c, off = 0;
        if (span & 1) {
            off += (rem % m->ns) * m->Nnu;
            rem /= m->ns;
        }
        for (int mm = m->M - 1; mm >= 0; --mm)
            if (span & (2 << mm)) {
                const int nm = rem % m->nb[mm];
                if (mm == m->M - 1) nlast[c] = nm;
                off += nm * m->stride[mm];
                rem /= m->nb[mm];
            }
        chain[c] = off;
    }
    for (int b = 0; b < bp.nblk; ++b) {
        int rem = b, off = 0;
        for (int mm = m->M - 1; mm >= 0; --mm)
            if (!(span & (2 << mm))) {
                off += (rem % m->nb[mm]) * m->stride[mm];
                rem /= m->nb[mm];
            }
        if (!(span & 1)) off += rem * m->Nnu;
        base[b] = off;
    }
    out->pd.L = bp.L;
    out->pd.nblk = bp.nblk;
    out->pd.p = bp.p;
    out->pd.span = span;
    out->pd.S = bp.S;
    out->pd.K = bp.K;
    out->wide = bp.wide;
    const bool last_in_chain = (span >> m->M) & 1;
    out->staged = false;
    if (last_in_chain) {
        for (int c = 0; c < bp.L; ++c)
            if (nlast[c] == 0) {
                run_c0.push_back(c);
                run_off.push_back(chain[c]);
            }
        out->pd.runlen = m->nb[m->M - 1];
        out->pd.nrun = (int)run_c0.size();
        out->pd.cs_run = (span & 1) ? m->ns : 1;
        const size_t tile = (size_t)bp.L * (32 + 1) * 16;  // worst case (FP64)
        out->staged = tile <= 160 * 1024 && bp.p <= PMAX;
        out->P = bp.p <= 2 ? 2 : bp.p <= 4 ? 4 : bp.p <= 8 ? 8 : 16;
    }
    if (run_c0.empty()) {
        run_c0.push_back(0);
        run_off.push_back(0);
    }
    const size_t n1 = chain.size(), n2 = base.size(), n3 = std::max<size_t>(1, bp.ent_dc.size()), n4 = run_off.size(),
                 n5 = run_c0.size(), n6 = bp.sw_combo.size();
    std::vector<int> all;
    all.reserve(n1 + n2 + n3 + n4 + n5 + n6);
    all.insert(all.end(), chain.begin(), chain.end());
    all.insert(all.end(), base.begin(), base.end());
    if (bp.ent_dc.empty())
        all.push_back(0);
    else
        all.insert(all.end(), bp.ent_dc.begin(), bp.ent_dc.end());
    all.insert(all.end(), run_off.begin(), run_off.end());
    all.insert(all.end(), run_c0.begin(), run_c0.end());
    all.insert(all.end(), bp.sw_combo.begin(), bp.sw_combo.end());
    VBK_CUDA(vbk_alloc(m, &out->mem, all.size() * sizeof(int), st));
    int* p = (int*)out->mem;
    VBK_CUDA(cudaMemcpyAsync(p, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    out->pd.chain_off = p;
    out->pd.fixed_base = p + n1;
    out->pd.ent_dc = p + n1 + n2;
    out->pd.run_off = p + n1 + n2 + n3;
    out->pd.run_c0 = p + n1 + n2 + n3 + n4;
    out->pd.swc = p + n1 + n2 + n3 + n4 + n5;
    out->pd.nswc = (int)(n6 / 5);
    // `all` must stay alive until the copy completes
    VBK_CUDA(cudaStreamSynchronize(st));
    return VBK_OK;
}

// Launches the block preconditioner z = B^-1 r (optionally fused with the COCG update).
template <class R> int prepare_staged(const DevPlanBuf& pb) {
    if (pb.wide) {
        if (pb.pd.S > LV_SMAX || 2 * (size_t)pb.pd.S * pb.pd.S * sizeof(cx<R>) > 220 * 1024) {
            vbk_set_error("block preconditioner band too wide for shared memory in this precision");
            return VBK_ERR_UNSUPPORTED;
        }
        return VBK_OK;
    }
    if (!pb.staged) return VBK_OK;
    const size_t smem = (size_t)pb.pd.L * (SG + 1) * sizeof(cx<R>);
    if (smem <= 48 * 1024) return VBK_OK;
    cudaError_t ce = cudaSuccess;
    switch (pb.P) {
        case 2: ce = cudaFuncSetAttribute(k_block_staged<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); break;
        case 4: ce = cudaFuncSetAttribute(k_block_staged<R, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); break;
        case 8: ce = cudaFuncSetAttribute(k_block_staged<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); break;
        default: ce = cudaFuncSetAttribute(k_block_staged<R, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); break;
    }
    return ce == cudaSuccess ? VBK_OK : vbk_cuda_fail(ce, "block preconditioner shared-memory opt-in");
}

template <class R>
void block_precond(Runner& rn, const DevPlanBuf& pb, int N, Sel sel, unsigned ny, const int* sys_e, const cx<R>* F,
                   const SysState* sst, int upd, cx<R>* x, cx<R>* r, long long rs, const cx<R>* p, const cx<R>* q, cx<R>* z,
                   long long zs, double2* part_rr, double2* part_rz);

inline unsigned cdiv_u(long long a, long long b);
// Opt the staged kernel of this plan in to the shared memory it needs (outside any capture).
template <class R> int prepare_staged(const DevPlanBuf& pb);

inline int block_partials(const DevPlanBuf& pb) {
    if (pb.wide) return pb.pd.nblk;
    return pb.staged ? (int)((pb.pd.nblk + 31) / 32) : (int)((pb.pd.nblk + BTPB - 1) / BTPB);
}


// Matvec variants (chosen per model and precision by the autotuner below):
//   0..3  register-blocked k_matvec3 with (S, EPT) = (1, 4), (2, 4), (4, 2), (2, 2)
//   4..7  windowed k_matvec_tiled with (S, EPT) = (1, 4), (2, 4), (4, 2), (8, 1)
//   8..9  direct k_matvec2 with S = 1, 4
//   10..11 one / two systems per CTA with x in shared memory (k_matvec_sys, FP32)
//   12..15 every state of a tile per CTA, windows staged by cp.async, coefficients from rows in
//          shared memory (k_matvec_win) with (S, EPT) = (2, 4), (2, 2), (4, 2), (1, 4)
//   16..19 persistent streaming kernel, tiles of rows of mode 0 brought in by bulk asynchronous
//          copies through a ring of shared-memory stages (k_matvec_stream, vbk_stream.cu)
constexpr int MV_NWIN = 16;  // variants 0..15 launched from this file
constexpr int MV_NVAR = VBK_MATVEC_NVARIANTS;
inline int mv_ept(int v) {
    static const int e[MV_NWIN] = {4, 4, 2, 2, 4, 4, 2, 1, 1, 1, 1, 1, 4, 2, 2, 4};
    return v < MV_NWIN ? e[v] : 1;
}
inline int mv_sys(int v) {
    static const int sv[MV_NWIN] = {1, 2, 4, 2, 1, 2, 4, 8, 1, 4, 1, 2, 2, 2, 4, 1};
    return v < MV_NWIN ? sv[v] : 1;
}
// window geometry of k_matvec_win: smallest in-plane offset and window length per state
inline void mv_win_geom(const DevModel& md, int v, int* lo, int* wst) {
    int l = 0, h = 0;
    for (int d = 0; d < md.ns; ++d) {
        l = std::min(l, md.lmin[d]);
        h = std::max(h, md.lmax[d]);
    }
    *lo = l;
    *wst = TPB * mv_ept(v) + h - l;
}
inline long long mv_win_smem(const DevModel& md, int v, size_t c) {
    int lo, wst;
    mv_win_geom(md, v, &lo, &wst);
    const long long wb = ((long long)mv_sys(v) * md.ns * wst * (long long)c + 15) & ~15LL;
    const long long rb = ((long long)md.nrct * 8 + 15) & ~15LL;
    return wb + rb + (long long)md.rbeg[md.ns] * 16;
}
inline int mv_window(const DevModel& md, int v) {
    int lr = 0;
    for (int d = 0; d < md.ns; ++d) lr = std::max(lr, md.lmax[d] - md.lmin[d]);
    return TPB * mv_ept(v) + lr;
}
inline int mv_tiled_smem(const DevModel& md, int v, size_t c) {
    if (v < 4 || v >= 8) return 0;
    if (md.ntab > MV_TAB_SMEM) return -1;  // the oscillator tables must fit the shared-memory copy
    const long long W = mv_window(md, v);
    const long long bytes = (long long)mv_sys(v) * md.ns * W * (long long)c + (long long)md.ntab * (long long)(c / 2) + 16;
    return bytes > 150 * 1024 ? -1 : (int)bytes;
}
inline bool mv_valid(const DevModel& md, int v, size_t c) {
    if (md.nsc) return v == 8;  // sandwich channels: k_sand_w + k_matvec_sw, launched in place of variant 8
    if (v >= MV_NWIN) {
        StreamPlan sp;
        return vbk_stream_plan(md, v - MV_NWIN, c, &sp);
    }
    if (v >= 12) return md.rok && mv_win_smem(md, v, c) <= 110 * 1024;
    if (v >= 10) return c == 8 && md.rok && matvec_sys_smem(md, v - 9) <= 220 * 1024;
    if (c == 16 && (mv_sys(v) * mv_ept(v) > 8 || v == 7)) return false;  // FP64: register budget
    return mv_tiled_smem(md, v, c) >= 0;
}
// partial sums per system that variant v writes for entries of c bytes (8: FP32, 16: FP64)
inline int matvec_partials_v(const DevModel& md, int v, size_t c) {
    if (md.nsc) v = 8;
    if (v >= MV_NWIN) {  // one partial per strip of the plan of this precision
        StreamPlan sp;
        return vbk_stream_plan(md, v - MV_NWIN, c, &sp) ? sp.nstrip : 1;
    }
    if (v >= 12) return (md.Nnu + TPB * mv_ept(v) - 1) / (TPB * mv_ept(v));  // one CTA per tile of all states
    if (v >= 10) return 1;
    const int T = TPB * mv_ept(v);
    return md.ns * ((md.Nnu + T - 1) / T);
}

template <class T, int S, int EPT>
void go_tiled(Runner& rn, const char* name, const DevModel& md, dim3 g, size_t smem, const int* sys_e, Sel sel,
              unsigned nlist, const cx<T>* diag, const cx<T>* x, long long xs, cx<T>* y, long long ys, const double2* b,
              double2* part, int red) {
    const int Wa = TPB * EPT + [&] {
        int lr = 0;
        for (int d = 0; d < md.ns; ++d) lr = std::max(lr, md.lmax[d] - md.lmin[d]);
        return lr;
    }();
    switch (md.M) {
        case 1: rn.go_smem(name, k_matvec_tiled<T, S, EPT, 1>, g, dim3(TPB), smem, md, Wa, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); break;
        case 2: rn.go_smem(name, k_matvec_tiled<T, S, EPT, 2>, g, dim3(TPB), smem, md, Wa, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); break;
        case 3: rn.go_smem(name, k_matvec_tiled<T, S, EPT, 3>, g, dim3(TPB), smem, md, Wa, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); break;
        default: rn.go_smem(name, k_matvec_tiled<T, S, EPT, 4>, g, dim3(TPB), smem, md, Wa, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); break;
    }
}

template <class T>
void launch_matvec_v(Runner& rn, int v, const char* name, const DevModel& md, const int* sys_e, Sel sel, unsigned nlist,
                     const cx<T>* diag, const cx<T>* x, long long xs, cx<T>* y, long long ys, const double2* b,
                     double2* part, int red) {
    if (md.nsc) {
        // q-dependent coupling: the two passes of the sandwich product (whatever variant was asked)
        if (nlist == 0) return;
        rn.go("sandwich_w", k_sand_w<T>, dim3(cdiv_u(md.Nnu, TPB), nlist), dim3(TPB), md, sys_e, sel, (int)nlist, x, xs);
        rn.go(name, k_matvec_sw<T>, dim3((unsigned)matvec_partials_v(md, 8, sizeof(cx<T>)), nlist), dim3(TPB), md, sys_e, sel, (int)nlist,
              diag, x, xs, y, ys, b, part, red);
        return;
    }
    if (v >= MV_NWIN) {
        StreamPlan sp;
        if (!vbk_stream_plan(md, v - MV_NWIN, sizeof(cx<T>), &sp)) {
            rn.note_error(cudaErrorInvalidConfiguration, name);
            return;
        }
        rn.go_custom(name, [&] {
            return vbk_stream_matvec(md, sp, sys_e, sel.list, sel.act, (int)nlist, diag, x, xs, y, ys, b, part, red,
                                     sizeof(T) == 4, rn.st);
        });
        return;
    }
    const int S = mv_sys(v);
    const dim3 g((unsigned)matvec_partials_v(md, v, sizeof(cx<T>)), (nlist + S - 1) / S);
    const size_t smem = (v >= 4 && v < 8) ? (size_t)mv_tiled_smem(md, v, sizeof(cx<T>)) : 0;
    if (v >= 12) {
        int lo, wst;
        mv_win_geom(md, v, &lo, &wst);
        const size_t sm = (size_t)mv_win_smem(md, v, sizeof(cx<T>));
        auto go = [&](auto kern) { rn.go_smem(name, kern, g, dim3(TPB), sm, md, lo, wst, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); };
        switch (v * 4 + md.M - 1) {
            case 48: go(k_matvec_win<T, 2, 4, 1>); break;
            case 49: go(k_matvec_win<T, 2, 4, 2>); break;
            case 50: go(k_matvec_win<T, 2, 4, 3>); break;
            case 51: go(k_matvec_win<T, 2, 4, 4>); break;
            case 52: go(k_matvec_win<T, 2, 2, 1>); break;
            case 53: go(k_matvec_win<T, 2, 2, 2>); break;
            case 54: go(k_matvec_win<T, 2, 2, 3>); break;
            case 55: go(k_matvec_win<T, 2, 2, 4>); break;
            case 56: go(k_matvec_win<T, 4, 2, 1>); break;
            case 57: go(k_matvec_win<T, 4, 2, 2>); break;
            case 58: go(k_matvec_win<T, 4, 2, 3>); break;
            case 59: go(k_matvec_win<T, 4, 2, 4>); break;
            case 60: go(k_matvec_win<T, 1, 4, 1>); break;
            case 61: go(k_matvec_win<T, 1, 4, 2>); break;
            case 62: go(k_matvec_win<T, 1, 4, 3>); break;
            default: go(k_matvec_win<T, 1, 4, 4>); break;
        }
        return;
    }
    if (v >= 10) {
        if constexpr (sizeof(T) == 4) {
            const int Sv = v - 9;
            const dim3 gs((nlist + Sv - 1) / Sv);
            const size_t sm = matvec_sys_smem(md, Sv);
            auto go = [&](auto kern) { rn.go_smem(name, kern, gs, dim3(RTPB), sm, md, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); };
            switch (md.M * 2 + (Sv - 1)) {
                case 2: go(k_matvec_sys<1, 1>); break;
                case 3: go(k_matvec_sys<1, 2>); break;
                case 4: go(k_matvec_sys<2, 1>); break;
                case 5: go(k_matvec_sys<2, 2>); break;
                case 6: go(k_matvec_sys<3, 1>); break;
                case 7: go(k_matvec_sys<3, 2>); break;
                case 8: go(k_matvec_sys<4, 1>); break;
                default: go(k_matvec_sys<4, 2>); break;
            }
        }
        return;
    }
    switch (v) {
        case 0: rn.go(name, k_matvec3<T, 1, 4>, g, dim3(TPB), md, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); break;
        case 1: rn.go(name, k_matvec3<T, 2, 4>, g, dim3(TPB), md, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); break;
        case 2: rn.go(name, k_matvec3<T, 4, 2>, g, dim3(TPB), md, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); break;
        case 3: rn.go(name, k_matvec3<T, 2, 2>, g, dim3(TPB), md, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); break;
        case 8: rn.go(name, k_matvec2<T, 1>, g, dim3(TPB), md, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); break;
        case 9: rn.go(name, k_matvec2<T, 4>, g, dim3(TPB), md, sys_e, sel, (int)nlist, diag, x, xs, y, ys, b, part, red); break;
        case 4: go_tiled<T, 1, 4>(rn, name, md, g, smem, sys_e, sel, nlist, diag, x, xs, y, ys, b, part, red); break;
        case 5: go_tiled<T, 2, 4>(rn, name, md, g, smem, sys_e, sel, nlist, diag, x, xs, y, ys, b, part, red); break;
        case 6: go_tiled<T, 4, 2>(rn, name, md, g, smem, sys_e, sel, nlist, diag, x, xs, y, ys, b, part, red); break;
        default:
            if constexpr (sizeof(T) == 4) go_tiled<T, 8, 1>(rn, name, md, g, smem, sys_e, sel, nlist, diag, x, xs, y, ys, b, part, red);
            break;
    }
}

// Opt the windowed variants in to the shared memory they need (outside any capture).
template <class T, int S, int EPT>
cudaError_t tiled_optin(const DevModel& md, int need) {
    switch (md.M) {
        case 1: return cudaFuncSetAttribute(k_matvec_tiled<T, S, EPT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        case 2: return cudaFuncSetAttribute(k_matvec_tiled<T, S, EPT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        case 3: return cudaFuncSetAttribute(k_matvec_tiled<T, S, EPT, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        default: return cudaFuncSetAttribute(k_matvec_tiled<T, S, EPT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    }
}
template <class T, int S, int EPT>
cudaError_t win_optin(const DevModel& md, int need) {
    switch (md.M) {
        case 1: return cudaFuncSetAttribute(k_matvec_win<T, S, EPT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        case 2: return cudaFuncSetAttribute(k_matvec_win<T, S, EPT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        case 3: return cudaFuncSetAttribute(k_matvec_win<T, S, EPT, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        default: return cudaFuncSetAttribute(k_matvec_win<T, S, EPT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    }
}
template <class T> int prepare_matvec(const DevModel& md) {
    if (const int rc = vbk_stream_prepare(md, sizeof(T) == 4)) return rc;
    const int need[4] = {mv_tiled_smem(md, 4, sizeof(cx<T>)), mv_tiled_smem(md, 5, sizeof(cx<T>)),
                         mv_tiled_smem(md, 6, sizeof(cx<T>)), mv_tiled_smem(md, 7, sizeof(cx<T>))};
    cudaError_t ce = cudaSuccess;
    for (int v = 12; v < 16 && ce == cudaSuccess; ++v) {
        if (!mv_valid(md, v, sizeof(cx<T>))) continue;
        const int sm = (int)mv_win_smem(md, v, sizeof(cx<T>));
        switch (v) {
            case 12: ce = win_optin<T, 2, 4>(md, sm); break;
            case 13: ce = win_optin<T, 2, 2>(md, sm); break;
            case 14: ce = win_optin<T, 4, 2>(md, sm); break;
            default: ce = win_optin<T, 1, 4>(md, sm); break;
        }
    }
    if (need[0] > 0) ce = tiled_optin<T, 1, 4>(md, need[0]);
    if (need[1] > 0 && ce == cudaSuccess) ce = tiled_optin<T, 2, 4>(md, need[1]);
    if (need[2] > 0 && ce == cudaSuccess) ce = tiled_optin<T, 4, 2>(md, need[2]);
    if constexpr (sizeof(T) == 4) {
        if (need[3] > 0 && ce == cudaSuccess) ce = tiled_optin<T, 8, 1>(md, need[3]);
        for (int Sv = 1; Sv <= 2 && ce == cudaSuccess; ++Sv) {
            if (!mv_valid(md, 9 + Sv, sizeof(cx<T>))) continue;
            const int sm = (int)matvec_sys_smem(md, Sv);
            auto opt = [&](auto kern) { return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm); };
            switch (md.M * 2 + (Sv - 1)) {
                case 2: ce = opt(k_matvec_sys<1, 1>); break;
                case 3: ce = opt(k_matvec_sys<1, 2>); break;
                case 4: ce = opt(k_matvec_sys<2, 1>); break;
                case 5: ce = opt(k_matvec_sys<2, 2>); break;
                case 6: ce = opt(k_matvec_sys<3, 1>); break;
                case 7: ce = opt(k_matvec_sys<3, 2>); break;
                case 8: ce = opt(k_matvec_sys<4, 1>); break;
                default: ce = opt(k_matvec_sys<4, 2>); break;
            }
        }
    }
    return ce == cudaSuccess ? VBK_OK : vbk_cuda_fail(ce, "matvec shared-memory opt-in");
}

// Autotuner: times every valid variant on the batch at hand (CUDA events, best of 3) and keeps
// the fastest for this model and precision.  Every variant writes the same y; the chosen one
// runs last so that the partials match its grid.
template <class T>
int tune_matvec(Runner& rn, vbk_model* mdl, const int* sys_e, Sel sel, unsigned nlist, const cx<T>* diag, const cx<T>* x,
                long long xs, cx<T>* y, long long ys, const double2* b, double2* part, int red) {
    const DevModel& md = mdl->dm;
    int& slot = mdl->mv_variant[sizeof(T) == 4 ? 0 : 1];
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return vbk_cuda_fail(cudaGetLastError(), "tuner");
    float best = 1e30f;
    int bestv = 0;
    const bool timing = rn.timing;
    rn.timing = false;
    for (int v = 0; v < MV_NVAR; ++v) {
        if (!mv_valid(md, v, sizeof(cx<T>))) continue;
        float tmin = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, rn.st);
            launch_matvec_v<T>(rn, v, "matvec_tune", md, sys_e, sel, nlist, diag, x, xs, y, ys, b, part, red);
            cudaEventRecord(e1, rn.st);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            tmin = std::min(tmin, ms);
        }
        if (tmin < best) {
            best = tmin;
            bestv = v;
        }
    }
    rn.timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    slot = bestv;
    if (timing) {  // the chosen variant's best time over the whole batch (one launch, all systems of the list)
        const int k = rn.id(sizeof(T) == 4 ? "matvec_tuned_fp32" : "matvec_tuned_fp64");
        mdl->timers[k].launches += 1;
        mdl->timers[k].ms += best;
    }
    launch_matvec_v<T>(rn, bestv, "matvec_tune", md, sys_e, sel, nlist, diag, x, xs, y, ys, b, part, red);
    if (const cudaError_t ce = cudaGetLastError(); ce != cudaSuccess) return vbk_cuda_fail(ce, "matvec tuner");
    return VBK_OK;
}

template <class T, int M>
void launch_matvec(Runner& rn, const char* name, const DevModel& md, const int* sys_e, Sel sel, unsigned nlist,
                   const cx<T>* diag, const cx<T>* x, long long xs, cx<T>* y, long long ys, const double2* b, double2* part,
                   int red, int variant) {
    launch_matvec_v<T>(rn, variant < 0 ? (sizeof(T) == 4 ? 1 : 3) : variant, name, md, sys_e, sel, nlist, diag, x, xs, y, ys, b,
                       part, red);
}
inline int matvec_partials(const DevModel& md, int variant, size_t c) { return matvec_partials_v(md, variant, c); }

// L D L^T factors of every block of every energy (Sec. III.B: computed once per energy and
// stored): thread-per-block kernel for narrow bands, band assembly + one CTA per block for
// wide ones.
template <class R, int M>
void factor_blocks(Runner& rn, const DevModel& md, const DevPlanBuf& pb, int nE, const cx<R>* diag, cx<R>* F, int* fail) {
    if (!pb.wide) {
        rn.go("block_factor", k_block_factor<R, M>, dim3(cdiv_u((long long)nE * pb.pd.nblk, 64)), dim3(64), md, pb.pd, nE,
              diag, F, fail);
        return;
    }
    const size_t smem = 2 * (size_t)pb.pd.S * pb.pd.S * sizeof(cx<R>);
    const cudaError_t ce = cudaFuncSetAttribute(k_level_factor<R, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        if (rn.first_error == cudaSuccess) rn.first_error = ce;
        vbk_set_error("level factorization shared-memory opt-in failed");
        return;
    }
    rn.go_smem("block_factor_wide", k_level_factor<R, M>, dim3(pb.pd.nblk, nE), dim3(LF_THREADS), smem, md, pb.pd, diag, F,
               fail);
}

template <class R, int M> struct Solver {
    static int run(vbk_model* mdl, const SolveJob& job, const vbk_opts& o, vbk_stats* stats, cudaStream_t st);
};

template <class R, int M>
int Solver<R, M>::run(vbk_model* mdl, const SolveJob& job, const vbk_opts& o, vbk_stats* stats, cudaStream_t st) {
    DevModel md = mdl->dm;  // own copy: the per-call buffers of q-dependent couplings are set below
    const int N = md.N, nsys = job.nsys, nE = job.nE;
    const bool mixed = sizeof(R) == 4;
    const int method = o.method;
    const int mres = std::max(1, std::min(o.restart, 256));
    const int pspan = o.precond_span;
    const bool block = pspan > 0;
    Runner rn{mdl, st, o.timing != 0, {}, {}};
    const bool sand = md.nsc > 0;  // q-dependent coupling (Sec. II.C)

    BlockPlan bp;
    DevPlanBuf pbuf;
    if (block) {
        int rc = vbk_make_block_plan(mdl, pspan, &bp);
        if (rc) return rc;
        rc = upload_plan(bp, mdl, st, &pbuf);
        if (!rc) rc = prepare_staged<R>(pbuf);
        if (rc) {
            if (pbuf.mem) cudaFreeAsync(pbuf.mem, st);
            return rc;
        }
    }

    {
        int rc = prepare_matvec<R>(md);
        if (!rc && sizeof(R) == 4) rc = prepare_matvec<double>(md);
        if (rc) {
            if (pbuf.mem) cudaFreeAsync(pbuf.mem, st);
            return rc;
        }
    }
    // a matvec variant the caller fixed for this solve: used for both operators (the Krylov
    // operator and the FP64 residual) where it is valid for their precision, in place of the
    // tuned choice; the model's tuned choices come back when the solve returns
    struct MvRestore {
        vbk_model* m;
        int v[2];
        bool on;
        ~MvRestore() {
            if (on) {
                m->mv_variant[0] = v[0];
                m->mv_variant[1] = v[1];
            }
        }
    } mv_restore{mdl, {mdl->mv_variant[0], mdl->mv_variant[1]}, o.matvec_variant >= 0};
    if (o.matvec_variant >= 0) {
        const int fv = o.matvec_variant;
        const bool ok_k = fv < MV_NVAR && mv_valid(md, fv, sizeof(cx<R>)), ok_64 = fv < MV_NVAR && mv_valid(md, fv, 16);
        if (!ok_k && !ok_64) {
            if (pbuf.mem) cudaFreeAsync(pbuf.mem, st);
            vbk_set_error("matvec variant not available for this model");
            return VBK_ERR_INVALID_ARG;
        }
        if (ok_k) mdl->mv_variant[sizeof(R) == 4 ? 0 : 1] = fv;
        if (ok_64) mdl->mv_variant[1] = fv;
    }
    const bool tune = o.autotune != 0 && !sand && o.matvec_variant < 0;
    // FP32 COCG with a point preconditioner and a system small enough for shared memory:
    // one CTA per system (k_cocg_resident)
    bool resident = sizeof(R) == 4 && method == VBK_COCG && pspan <= 0 && !sand && resident_ok(md) && o.resident != 0;
    if (resident && prepare_resident<M>(md) != VBK_OK) {
        cudaGetLastError();
        resident = false;
    }
    // The resident FP32 path refines in double-float arithmetic: the solution accumulates as
    // (hi, lo) float pairs and b - A x is formed on the FP32 pipes (k_residual_df); psi is
    // converted to FP64 once at the end.
    const bool dfr = resident;
    // the double-float residual with one CTA per system when the split solution fits shared memory
    const bool dfr_res = dfr && prepare_residual_res<M>(md);
    const bool spec = dfr_res && o.timing == 0;  // refinement rounds enqueued ahead of the host check
    // The whole refinement of every system in one launch: resident = 1, one CTA per system
    // (k_solve_resident); resident = 3, one cluster of n_s CTAs per system (vbk_cluster.cu)
    ClArgs cla;
    size_t cl_smem = 0;
    int cl_n = 0;
    int fused = 0;
    if (resident && o.resident == 1 && prepare_solve_resident<M>(md)) fused = 1;
    if (resident && o.resident == 3 && vbk_cluster_plan(md, &cla, &cl_smem)) {
        if (vbk_cluster_prepare(md, cla, cl_smem, &cl_n) == VBK_OK && cl_n >= 1)
            fused = 2;
        else
            cudaGetLastError();
    }
    const bool cluster = fused != 0;

    // ---- workspace
    const size_t NN = (size_t)N;
    const int nb_e = (int)cdiv_u(N, TPB);       // element-wise kernels
    int nb_mv = matvec_partials(md, mdl->mv_variant[sizeof(R) == 4 ? 0 : 1] < 0 ? 0 : mdl->mv_variant[sizeof(R) == 4 ? 0 : 1],
                                sizeof(cx<R>));
    int nb_mv_max = 0;  // the largest partial count of any variant
    for (int v = 0; v < MV_NVAR; ++v)  // either precision: the FP64 residual shares the buffers
        nb_mv_max = std::max(nb_mv_max, std::max(matvec_partials(md, v, 8), matvec_partials(md, v, 16)));
    const int nb_v = (int)cdiv_u(N, VCHUNK);    // basis-vector kernels
    const int nb_b = block ? block_partials(pbuf) : 0;
    const int nslot = std::max(std::max(nb_e, nb_mv_max), std::max(nb_b, nb_v * (mres + 1)));
    size_t bytes = 0;
    bytes += carve_size<double2>(dfr ? 1 : (size_t)nE * NN);         // diag64 (diagonal split in df mode)
    if (dfr) bytes += carve_size<float4>((size_t)nE * NN) + 2 * carve_size<float4>((size_t)nsys * NN);  // dsp, xs, rs
    bytes += carve_size<cx<R>>(mixed ? (size_t)nE * NN : 1);          // diagR
    bytes += carve_size<float2>(mixed ? (size_t)nE * NN : 1);         // 1/diag (FP32)
    bytes += carve_size<double2>((size_t)nsys * NN);                  // r64
    bytes += carve_size<SysState>(nsys);
    // energies and the per-system index arrays set from the host: one block, one copy
    const size_t small_bytes = (size_t)nE * sizeof(double) + 5 * (size_t)nsys * sizeof(int);
    bytes += carve_size<char>(small_bytes);
    bytes += 3 * carve_size<int>(nsys) + carve_size<int>(nE) + carve_size<int>(4);
    bytes += 3 * carve_size<double2>((size_t)nsys * nslot);           // partial buffers
    if (block) bytes += carve_size<cx<R>>((size_t)nE * factor_entries(bp, NN));
    const size_t n_g = sand ? (size_t)nE * md.npair * md.Nnu : 1, n_w = sand ? (size_t)nsys * md.nsc * md.Nnu : 1;
    if (sand) {  // pair tables, sandwich diagonal, inner-pass vectors w (FP64 size, shared by the FP32 pass)
        bytes += carve_size<double2>(n_g) + carve_size<float2>(mixed ? n_g : 1);
        bytes += carve_size<double2>((size_t)nE * NN) + carve_size<float2>(mixed ? (size_t)nE * NN : 1);
        bytes += carve_size<double2>(n_w);
    }
    if (method == VBK_COCG) {
        bytes += 5 * carve_size<cx<R>>((size_t)nsys * NN);            // x r p q z
    } else {
        bytes += carve_size<cx<R>>((size_t)nsys * NN * (mres + 1));   // V
        bytes += 2 * carve_size<cx<R>>((size_t)nsys * NN);            // z, w
        bytes += carve_size<double2>((size_t)nsys * (mres + 1) * mres);  // H
        bytes += 4 * carve_size<double2>((size_t)nsys * (mres + 1));     // g, h1, h2, y
        bytes += carve_size<double2>((size_t)nsys * mres);               // sn
        bytes += carve_size<double>((size_t)nsys * mres);                // cs
        bytes += carve_size<double>((size_t)nsys);                       // inv_h
    }
    char* wsbase = nullptr;
    {
        cudaError_t e = vbk_alloc(mdl, (void**)&wsbase, bytes, st);
        if (e != cudaSuccess) {
            if (pbuf.mem) cudaFreeAsync(pbuf.mem, st);
            vbk_set_error("workspace allocation of " + std::to_string(bytes) + " bytes failed");
            cudaGetLastError();
            return VBK_ERR_OOM;
        }
    }
    char* p = wsbase;
    double2* diag64 = carve<double2>(p, dfr ? 1 : (size_t)nE * NN);
    float4 *dsp = nullptr, *xs = nullptr, *rsp = nullptr;
    if (dfr) {
        dsp = carve<float4>(p, (size_t)nE * NN);
        xs = carve<float4>(p, (size_t)nsys * NN);
        rsp = carve<float4>(p, (size_t)nsys * NN);
    }
    cx<R>* diagR = carve<cx<R>>(p, mixed ? (size_t)nE * NN : 1);
    if (!mixed) diagR = reinterpret_cast<cx<R>*>(diag64);
    float2* dinvR = carve<float2>(p, mixed ? (size_t)nE * NN : 1);
    if (!mixed) dinvR = nullptr;
    double2* r64 = carve<double2>(p, (size_t)nsys * NN);
    SysState* sst = carve<SysState>(p, nsys);
    char* smallp = carve<char>(p, small_bytes);
    double* dE = reinterpret_cast<double*>(smallp);
    int* sys_e = reinterpret_cast<int*>(smallp + (size_t)nE * sizeof(double));
    int* outer = sys_e + nsys;
    int* alll = outer + nsys;
    int* olist = alll + nsys;
    int* ilist = olist + nsys;
    int* inner = carve<int>(p, nsys);
    int* ilist2 = carve<int>(p, nsys);  // second list of the persistent COCG iterations
    int* done = carve<int>(p, nsys);    // per-system work-item counters (self-resetting)
    int* pfail = carve<int>(p, nE);
    int* cnt = carve<int>(p, 4);
    double2* partA = carve<double2>(p, (size_t)nsys * nslot);
    double2* partB = carve<double2>(p, (size_t)nsys * nslot);
    double2* partC = carve<double2>(p, (size_t)nsys * nslot);
    cx<R>* F = block ? carve<cx<R>>(p, (size_t)nE * factor_entries(bp, NN)) : nullptr;
    if (sand) {
        md.sg64 = carve<double2>(p, n_g);
        md.sg32 = carve<float2>(p, mixed ? n_g : 1);
        md.sfd64 = carve<double2>(p, (size_t)nE * NN);
        md.sfd32 = carve<float2>(p, mixed ? (size_t)nE * NN : 1);
        md.sw64 = carve<double2>(p, n_w);
        md.sw32 = reinterpret_cast<float2*>(md.sw64);  // the FP32 and FP64 passes never overlap
        if (!mixed) md.sg32 = nullptr, md.sfd32 = nullptr;
    }
    cx<R>*x = nullptr, *r = nullptr, *pv = nullptr, *q = nullptr, *z = nullptr, *V = nullptr, *w = nullptr;
    double2 *H = nullptr, *g = nullptr, *h1 = nullptr, *h2 = nullptr, *yv = nullptr, *sn = nullptr;
    double *cs = nullptr, *invh = nullptr;
    if (method == VBK_COCG) {
        x = carve<cx<R>>(p, (size_t)nsys * NN);
        r = carve<cx<R>>(p, (size_t)nsys * NN);
        pv = carve<cx<R>>(p, (size_t)nsys * NN);
        q = carve<cx<R>>(p, (size_t)nsys * NN);
        z = carve<cx<R>>(p, (size_t)nsys * NN);
    } else {
        V = carve<cx<R>>(p, (size_t)nsys * NN * (mres + 1));
        z = carve<cx<R>>(p, (size_t)nsys * NN);
        w = carve<cx<R>>(p, (size_t)nsys * NN);
        H = carve<double2>(p, (size_t)nsys * (mres + 1) * mres);
        g = carve<double2>(p, (size_t)nsys * (mres + 1));
        h1 = carve<double2>(p, (size_t)nsys * (mres + 1));
        h2 = carve<double2>(p, (size_t)nsys * (mres + 1));
        yv = carve<double2>(p, (size_t)nsys * (mres + 1));
        sn = carve<double2>(p, (size_t)nsys * mres);
        cs = carve<double>(p, (size_t)nsys * mres);
        invh = carve<double>(p, (size_t)nsys);
    }

    int rc = VBK_OK;
    cudaGraphExec_t gexec = nullptr, pgexec = nullptr;
    long long p_per_launch = 0;
    // pinned staging (model-owned, reused): [host counters | set-up block | per-system states]
    const size_t o_stage = 256, o_hst = o_stage + ((small_bytes + 255) & ~size_t(255));
    char* hp = static_cast<char*>(vbk_pinned(mdl, o_hst + (size_t)nsys * sizeof(SysState)));
    int* hcnt = reinterpret_cast<int*>(hp);
    SysState* hst = hp ? reinterpret_cast<SysState*>(hp + o_hst) : nullptr;
    auto fail = [&](int code) {
        rc = code;
        return code;
    };
    do {
        if (!hp) {
            vbk_set_error("pinned host staging buffer allocation failed");
            fail(VBK_ERR_OOM);
            break;
        }
        {
            char* stage = hp + o_stage;
            std::memcpy(stage, job.E.data(), (size_t)nE * sizeof(double));
            int* si = reinterpret_cast<int*>(stage + (size_t)nE * sizeof(double));
            std::memcpy(si, job.sys_e.data(), (size_t)nsys * sizeof(int));
            for (int k = 0; k < nsys; ++k) {
                si[nsys + k] = 1;      // outer
                si[2 * nsys + k] = k;  // all systems
                si[3 * nsys + k] = k;  // outer list
                si[4 * nsys + k] = k;  // inner list
            }
        }
        if (cudaMemcpyAsync(smallp, hp + o_stage, small_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(sst, 0, nsys * sizeof(SysState), st) != cudaSuccess ||
            // (the one-CTA fused solve writes its split solution before reading it)
            (fused != 1 && cudaMemsetAsync(dfr ? (void*)xs : (void*)job.x64, 0, (size_t)nsys * NN * sizeof(double2), st) !=
                               cudaSuccess) ||
            cudaMemsetAsync(pfail, 0, nE * sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync(done, 0, nsys * sizeof(int), st) != cudaSuccess) {
            fail(vbk_cuda_fail(cudaGetLastError(), "solver set-up copies"));
            break;
        }
        // energy tables (FP64 + inner-precision copy); pair transforms of q-dependent couplings first
        if (sand) rn.go("sandwich_table", k_sand_table, dim3(cdiv_u(md.Nnu, TPB), nE), dim3(TPB), md, nE, (const double*)dE);
        if (dfr)  // the resident FP32 paths: double-float tables on the FP32 pipes
            rn.go("diag_table", k_diag_table_df, dim3(cdiv_u(N, TPB), nE), dim3(TPB), md, nE, (const double*)dE,
                  reinterpret_cast<float2*>(diagR), dinvR, dsp, pspan == 0 ? pfail : (int*)nullptr);
        else
            rn.go("diag_table", k_diag_table<M>, dim3(cdiv_u(N, TPB), nE), dim3(TPB), md, nE, (const double*)dE, diag64,
                  mixed ? reinterpret_cast<float2*>(diagR) : (float2*)nullptr, dinvR, (float4*)nullptr,
                  pspan == 0 ? pfail : (int*)nullptr);
        if (block) factor_blocks<R, M>(rn, md, pbuf, nE, (const cx<R>*)diagR, F, pfail);
        if (cudaError_t ce = cudaGetLastError(); ce != cudaSuccess) {
            fail(vbk_cuda_fail(ce, "set-up kernels"));
            break;
        }
        if (rn.first_error != cudaSuccess) {
            fail(VBK_ERR_CUDA);
            break;
        }
        const unsigned gs = cdiv_u(nsys, 128);
        const unsigned gw = cdiv_u(nsys, 4);  // warp-per-system kernels, 4 warps per block
        const int pmode = pspan < 0 ? -1 : (block ? 1 : 0);
        unsigned n_out = (unsigned)nsys;  // systems in olist (host copy)
        unsigned n_in = (unsigned)nsys;   // upper bound of systems in ilist
        // z = B^-1 src for the systems of `sel` (+ optional r^T z partials)
        auto precond = [&](Sel sel, unsigned ny, const cx<R>* src, long long ss, cx<R>* dst, long long ds, double2* part) {
            if (block)
                block_precond<R>(rn, pbuf, N, sel, ny, (const int*)sys_e, (const cx<R>*)F, (const SysState*)sst, 0, nullptr,
                                 const_cast<cx<R>*>(src), ss, nullptr, nullptr, dst, ds, nullptr, part);
            else
                rn.go("point_precond", k_point_precond<R>, dim3(nb_e, ny), dim3(TPB), N, (const int*)sys_e, sel, pmode,
                      (const cx<R>*)diagR, src, ss, dst, ds, part);
        };
        const int nb_rz = block ? nb_b : nb_e;

        if (cluster) {
            cla.nsys = nsys;
            cla.pmode = pmode;
            cla.max_refine = o.max_refine;
            cla.max_iter = o.max_iter;
            cla.inner_cap = o.inner_max_iter;
            cla.stall_check = 1;
            cla.tol = o.tol;
            cla.inner_tol = o.inner_tol;
            cla.counter = cnt;
            cla.sys_e = sys_e;
            cla.diag32 = reinterpret_cast<const float2*>(diagR);
            cla.diagdf = dsp;
            cla.b64 = job.b64;
            cla.bn2 = job.bnorm2;
            cla.xs = xs;
            cla.psi = job.x64;
            cla.st = sst;
            set_quad_args(md, M, cla);
            if (cudaMemsetAsync(cnt, 0, sizeof(int), st) != cudaSuccess) {
                fail(vbk_cuda_fail(cudaGetLastError(), "cluster solve set-up"));
                break;
            }
            if (fused == 1) {
                static int nsm = 0;
                if (nsm == 0 && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) nsm = 148;
                const dim3 g((unsigned)std::min(nsys, nsm));
                const SolveResidentFn kern = solve_resident_fn<M>(md);
                rn.go_smem("solve_resident", kern, g, dim3(RTPB), solve_resident_smem(md), md, cla,
                           reinterpret_cast<float2*>(x), reinterpret_cast<float2*>(r), (const float2*)dinvR);
            } else {
                rn.go_custom("solve_cluster", [&] { return vbk_cluster_launch(md, cla, cl_smem, std::min(cl_n, nsys), st); });
            }
            if (rn.first_error != cudaSuccess) {
                fail(VBK_ERR_CUDA);
                break;
            }
        }
        for (int it = 0; !cluster && it <= o.max_refine + 1; ++it) {
            // FP64 residual r = b - A x
            const Sel so{olist, outer};
            // the first residual is b itself (x = 0): only its norm is computed, and the first
            // inner solve reads b directly
            if (it == 0) {
                if (!job.bnorm2) rn.go("rhs_norm", k_rhs_norm, dim3(nsys), dim3(TPB), N, job.b64, partA);
            }
            else if (dfr_res)
                rn.go_smem("residual_df", k_residual_res<M>, dim3(n_out), dim3(RTPB), residual_res_smem(md), md,
                           (const int*)sys_e, (const int*)olist, (const float4*)dsp, (const float4*)xs, job.b64, rsp, partA);
            else if (dfr)
                rn.go("residual_df", k_residual_df<DF_S, DF_EPT>,
                      dim3(df_partials(md), cdiv_u(n_out, DF_S)), dim3(TPB), md, (const int*)sys_e, so, (int)n_out,
                      (const float4*)dsp, (const float4*)xs, job.b64, rsp, partA);
            else
            {
                if (tune && mdl->mv_variant[1] < 0) {
                    if (int trc = tune_matvec<double>(rn, mdl, (const int*)sys_e, so, n_out, (const double2*)diag64,
                                                      (const double2*)job.x64, (long long)N, r64, (long long)N, job.b64,
                                                      partA, 2)) {
                        fail(trc);
                        break;
                    }
                } else {
                    launch_matvec<double, M>(rn, "matvec_fp64", md, (const int*)sys_e, so, n_out, (const double2*)diag64,
                                             (const double2*)job.x64, (long long)N, r64, (long long)N, job.b64, partA, 2,
                                             mdl->mv_variant[1]);
                }
            }
            cudaMemsetAsync(cnt, 0, 4 * sizeof(int), st);
            cudaMemsetAsync(olist, 0xff, nsys * sizeof(int), st);  // -1: no system
            cudaMemsetAsync(ilist, 0xff, nsys * sizeof(int), st);
            rn.go("outer_check", k_outer_check, dim3(gs), dim3(128), nsys, sst, outer, inner, (const double2*)partA,
                  it == 0 || dfr_res ? 1 : dfr ? df_partials(md) : matvec_partials(md, mdl->mv_variant[1] < 0 ? 3 : mdl->mv_variant[1], 16),
                  it == 0 ? job.bnorm2 : (const double*)nullptr, it == 0 ? 1 : 0, o.tol, mixed ? o.inner_tol : 0.0, o.max_refine, o.max_iter,
                  mixed && method == VBK_COCG ? o.inner_max_iter : 0, mixed && method == VBK_COCG ? 1 : 0, cnt, olist,
                  ilist);
            if (resident && nsys <= ORDER_MAX)  // longest expected inner solve first (one CTA each)
                rn.go("order_lists", k_order_lists, dim3(1), dim3(1024), nsys, (const SysState*)sst, (const int*)inner, olist,
                      ilist);
            cudaMemcpyAsync(hcnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (spec && it < 2) {
                // the first two refinement rounds are enqueued without waiting for the count:
                // the one-CTA-per-system kernels run over every list slot and slots past the
                // count (-1) return at once; a solve takes at least two inner solves
                n_out = n_in = (unsigned)nsys;
            } else {
                if (cudaStreamSynchronize(st) != cudaSuccess) {
                    fail(vbk_cuda_fail(cudaGetLastError(), "outer check"));
                    break;
                }
                rn.flush();
                if (hcnt[0] == 0) break;
                n_out = n_in = (unsigned)hcnt[0];
            }
            const Sel si{ilist, inner};
            const Sel so2{olist, outer};

            const double2* res = it == 0 ? job.b64 : (const double2*)r64;  // the current FP64 residual
            if (method == VBK_COCG && resident && !block) {
                // one CTA per system runs the whole inner solve: scaled double-float residual in,
                // double-float correction out (list = ilist from the outer check)
                auto res_go = [&](auto kern) {
                    rn.go_smem("cocg_resident", kern, dim3(n_in), dim3(RTPB), resident_smem(md), md,
                               (const int*)sys_e, (const int*)ilist, pmode, reinterpret_cast<const float2*>(diagR),
                               (const float2*)dinvR, reinterpret_cast<float2*>(x), reinterpret_cast<float2*>(r),
                               it == 0 ? job.b64 : (const double2*)nullptr, (const float4*)rsp, xs, sst, inner, outer,
                               o.max_iter);
                };
                if (md.rsec)
                    res_go(k_cocg_resident<M, true>);
                else
                    res_go(k_cocg_resident<M, false>);
            } else if (method == VBK_COCG) {
                // r = rhs, x = 0, z = B^-1 r, p = z, rho = r^T z.  With a block preconditioner the
                // search direction carries over from the previous inner solve (k_cocg_start):
                // hard problems (thousands of iterations) then keep their Krylov progress across
                // the FP64 residual refreshes instead of restarting.
                rn.go("inner_rhs", k_inner_rhs<R>, dim3(nb_e, n_in), dim3(TPB), N, si, (const SysState*)sst, res, r,
                      (long long)N);
                cudaMemsetAsync(x, 0, (size_t)nsys * NN * sizeof(cx<R>), st);
                precond(si, n_in, r, N, z, N, partB);
                rn.go("cocg_start", k_cocg_start, dim3(gs), dim3(128), nsys, sst, (const int*)inner, (const double2*)partB,
                      nb_rz, block ? 1 : 0);
                if (block) {
                    if (it == 0) cudaMemsetAsync(pv, 0, (size_t)nsys * NN * sizeof(cx<R>), st);
                    rn.go("cocg_p", k_cocg_p<R>, dim3(nb_e, n_in), dim3(TPB), N, si, (const SysState*)sst, (const cx<R>*)z,
                          pv);
                } else {
                    cudaMemcpyAsync(pv, z, (size_t)nsys * NN * sizeof(cx<R>), cudaMemcpyDeviceToDevice, st);
                }
                if (tune && mdl->mv_variant[sizeof(R) == 4 ? 0 : 1] < 0) {
                    if (int trc = tune_matvec<R>(rn, mdl, (const int*)sys_e, si, n_in, (const cx<R>*)diagR, (const cx<R>*)pv,
                                                 (long long)N, q, (long long)N, (const double2*)nullptr, partA, 1)) {
                        fail(trc);
                        break;
                    }
                }
                const int mvv = mdl->mv_variant[sizeof(R) == 4 ? 0 : 1];
                nb_mv = matvec_partials(md, mvv < 0 ? (sizeof(R) == 4 ? 1 : 3) : mvv, sizeof(cx<R>));
                // one COCG iteration for the systems of the inner list
                auto cocg_iter = [&](unsigned ny) {
                    const Sel sc{ilist, inner};
                    launch_matvec<R, M>(rn, "matvec", md, (const int*)sys_e, sc, ny, (const cx<R>*)diagR, (const cx<R>*)pv,
                                        (long long)N, q, (long long)N, (const double2*)nullptr, partA, 1, mvv);
                    rn.go("cocg_alpha", k_cocg_alpha, dim3(gw), dim3(128), nsys, sst, inner, outer, (const double2*)partA,
                          nb_mv);
                    if (block) {
                        // fused x += alpha p, r -= alpha q and z = B^-1 r
                        block_precond<R>(rn, pbuf, N, sc, ny, (const int*)sys_e, (const cx<R>*)F, (const SysState*)sst, 1, x,
                                         r, (long long)N, (const cx<R>*)pv, (const cx<R>*)q, z, (long long)N, partC, partB);
                    } else {
                        rn.go("cocg_update", k_cocg_update<R>, dim3(nb_e, ny), dim3(TPB), N, sc, (const SysState*)sst,
                              (const int*)sys_e, pmode, (const cx<R>*)diagR, x, r, (const cx<R>*)pv, (const cx<R>*)q, z,
                              partC, partB);
                    }
                    cudaMemsetAsync(cnt, 0, sizeof(int), rn.st);
                    cudaMemsetAsync(ilist, 0xff, nsys * sizeof(int), rn.st);
                    rn.go("cocg_beta", k_cocg_beta, dim3(gw), dim3(128), nsys, sst, inner, outer, (const double2*)partC,
                          (block && pbuf.staged) ? nb_rz : nb_e, (const double2*)partB, nb_rz, o.max_iter, cnt, ilist);
                    rn.go("cocg_p", k_cocg_p<R>, dim3(nb_e, ny), dim3(TPB), N, sc, (const SysState*)sst, (const cx<R>*)z, pv);
                };
                const int K = std::max(1, o.check_every);
                int k = 0;
                if (!block && !sand) {
                    // persistent iterations: static grids over the device-side lists (A = ilist with
                    // count cnt[0], B = ilist2 with count cnt[1]); K (even) iterations per CUDA graph,
                    // captured once per solve and relaunched until list A is empty.  With timing on,
                    // the same kernels are launched directly (an event pair each).
                    const int K2 = K + (K & 1);
                    int sms = 0;
                    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, mdl->device);
                    if (sms <= 0) sms = 148;
                    auto grid_of = [&](auto kern) {
                        int nb = 0;
                        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, TPB, 0);
                        return (unsigned)(std::max(1, nb) * sms);
                    };
                    const int v = mvv;
                    const int pS = (v == 0) ? 1 : (v == 2) ? 4 : 2, pE = (v == 0 || v == 1) ? 4 : 2;
                    const unsigned g_mv = pS == 1   ? grid_of(k_pmatvec<R, 1, 4>)
                                          : pS == 4 ? grid_of(k_pmatvec<R, 4, 2>)
                                          : pE == 4 ? grid_of(k_pmatvec<R, 2, 4>)
                                                    : grid_of(k_pmatvec<R, 2, 2>);
                    const unsigned g_up = grid_of(k_pupdate<R, 8>), g_pp = grid_of(k_pp<R, 4>);
                    // mvname: the first matvec of an inner solve (every system of the inner list
                    // active) is timed under its own name when timing is on
                    auto piter = [&](int t, const char* mvname = "matvec") {
                        const DList cur{t % 2 == 0 ? ilist : ilist2, cnt + (t % 2)};
                        const DList nxt{t % 2 == 0 ? ilist2 : ilist, cnt + 1 - (t % 2)};
                        cudaMemsetAsync(cnt + 1 - (t % 2), 0, sizeof(int), rn.st);
                        if (pS == 1)
                            rn.go(mvname, k_pmatvec<R, 1, 4>, dim3(g_mv), dim3(TPB), md, (const int*)sys_e, cur,
                                  (const cx<R>*)diagR, (const cx<R>*)pv, q, partA, done, sst, inner, outer);
                        else if (pS == 4)
                            rn.go(mvname, k_pmatvec<R, 4, 2>, dim3(g_mv), dim3(TPB), md, (const int*)sys_e, cur,
                                  (const cx<R>*)diagR, (const cx<R>*)pv, q, partA, done, sst, inner, outer);
                        else if (pE == 4)
                            rn.go(mvname, k_pmatvec<R, 2, 4>, dim3(g_mv), dim3(TPB), md, (const int*)sys_e, cur,
                                  (const cx<R>*)diagR, (const cx<R>*)pv, q, partA, done, sst, inner, outer);
                        else
                            rn.go(mvname, k_pmatvec<R, 2, 2>, dim3(g_mv), dim3(TPB), md, (const int*)sys_e, cur,
                                  (const cx<R>*)diagR, (const cx<R>*)pv, q, partA, done, sst, inner, outer);
                        rn.go("cocg_update", k_pupdate<R, 8>, dim3(g_up), dim3(TPB), N, (const int*)sys_e, cur, pmode,
                              (const cx<R>*)diagR, x, r, (const cx<R>*)pv, (const cx<R>*)q, z, partC, partB, done, sst, inner,
                              outer, o.max_iter, (int*)nxt.list, (int*)nxt.count);
                        rn.go("cocg_p", k_pp<R, 4>, dim3(g_pp), dim3(TPB), N, nxt, (const SysState*)sst, (const cx<R>*)z, pv);
                    };
                    if (!rn.timing && !pgexec) {
                        const long long l0 = mdl->launches;
                        if (!mdl->cap_stream &&
                            cudaStreamCreateWithFlags(&mdl->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
                            fail(vbk_cuda_fail(cudaGetLastError(), "capture stream"));
                            break;
                        }
                        if (cudaStreamBeginCapture(mdl->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                            fail(vbk_cuda_fail(cudaGetLastError(), "graph capture"));
                            break;
                        }
                        rn.st = mdl->cap_stream;
                        for (int t = 0; t < K2; ++t) piter(t);
                        rn.st = st;
                        cudaGraph_t graph = nullptr;
                        const cudaError_t ce = cudaStreamEndCapture(mdl->cap_stream, &graph);
                        p_per_launch = mdl->launches - l0;
                        mdl->launches = l0;
                        if (ce != cudaSuccess || rn.first_error != cudaSuccess) {
                            if (graph) cudaGraphDestroy(graph);
                            fail(ce != cudaSuccess ? vbk_cuda_fail(ce, "graph capture") : VBK_ERR_CUDA);
                            break;
                        }
                        if (cudaGraphInstantiate(&pgexec, graph, 0) != cudaSuccess) {
                            cudaGraphDestroy(graph);
                            pgexec = nullptr;
                            fail(vbk_cuda_fail(cudaGetLastError(), "graph instantiation"));
                            break;
                        }
                        cudaGraphDestroy(graph);
                    }
                    for (;;) {
                        if (rn.timing) {
                            for (int t = 0; t < K2; ++t) piter(t, k == 0 && t == 0 ? "matvec_full" : "matvec");
                        } else {
                            if (cudaGraphLaunch(pgexec, st) != cudaSuccess) {
                                fail(vbk_cuda_fail(cudaGetLastError(), "graph launch"));
                                break;
                            }
                            mdl->launches += p_per_launch;
                        }
                        k += K2;
                        cudaMemcpyAsync(hcnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
                        if (cudaStreamSynchronize(st) != cudaSuccess) {
                            fail(vbk_cuda_fail(cudaGetLastError(), "COCG iterations"));
                            break;
                        }
                        rn.flush();
                        if (hcnt[0] == 0 || k > o.max_iter + K2) break;
                    }
                } else if (!rn.timing) {
                    // K iterations as one CUDA graph (grids sized for the active systems; systems that
                    // retire inside a chunk leave their CTAs at once), relaunched until none is active and
                    // re-captured when the active count has halved
                    long long per_launch = 0;
                    auto capture = [&](unsigned ny) -> bool {
                        // captured on a library-owned stream (the caller's may be the legacy default stream,
                        // which cannot be captured); the graph is launched on the caller's stream
                        if (!mdl->cap_stream &&
                            cudaStreamCreateWithFlags(&mdl->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
                            fail(vbk_cuda_fail(cudaGetLastError(), "capture stream"));
                            return false;
                        }
                        const long long l0 = mdl->launches;
                        if (cudaStreamBeginCapture(mdl->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                            fail(vbk_cuda_fail(cudaGetLastError(), "graph capture"));
                            return false;
                        }
                        rn.st = mdl->cap_stream;
                        for (int t = 0; t < K; ++t) cocg_iter(ny);
                        rn.st = st;
                        cudaGraph_t graph = nullptr;
                        const cudaError_t ce = cudaStreamEndCapture(mdl->cap_stream, &graph);
                        per_launch = mdl->launches - l0;
                        mdl->launches = l0;
                        if (ce != cudaSuccess || rn.first_error != cudaSuccess) {
                            if (graph) cudaGraphDestroy(graph);
                            fail(ce != cudaSuccess ? vbk_cuda_fail(ce, "graph capture") : VBK_ERR_CUDA);
                            return false;
                        }
                        bool ok = false;
                        if (gexec) {
                            cudaGraphExecUpdateResultInfo info;
                            ok = cudaGraphExecUpdate(gexec, graph, &info) == cudaSuccess;
                            if (!ok) {
                                cudaGetLastError();
                                cudaGraphExecDestroy(gexec);
                                gexec = nullptr;
                            }
                        }
                        if (!ok && cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) {
                            cudaGraphDestroy(graph);
                            gexec = nullptr;
                            fail(vbk_cuda_fail(cudaGetLastError(), "graph instantiation"));
                            return false;
                        }
                        cudaGraphDestroy(graph);
                        return true;
                    };
                    unsigned ny = n_in;
                    if (!capture(ny)) break;
                    for (;;) {
                        if (cudaGraphLaunch(gexec, st) != cudaSuccess) {
                            fail(vbk_cuda_fail(cudaGetLastError(), "graph launch"));
                            break;
                        }
                        mdl->launches += per_launch;
                        k += K;
                        cudaMemcpyAsync(hcnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
                        if (cudaStreamSynchronize(st) != cudaSuccess) {
                            fail(vbk_cuda_fail(cudaGetLastError(), "COCG iterations"));
                            break;
                        }
                        if (hcnt[0] == 0 || k > o.max_iter + K) break;
                        if ((unsigned)hcnt[0] * 2 <= ny) {
                            ny = (unsigned)hcnt[0];
                            if (!capture(ny)) break;
                        }
                    }
                } else {
                    for (;;) {
                        cocg_iter(n_in);
                        ++k;
                        if (k % K == 0) {
                            cudaMemcpyAsync(hcnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
                            if (cudaStreamSynchronize(st) != cudaSuccess) {
                                fail(vbk_cuda_fail(cudaGetLastError(), "COCG iterations"));
                                break;
                            }
                            rn.flush();
                            if (hcnt[0] == 0) break;
                            n_in = (unsigned)hcnt[0];
                        }
                        if (k > o.max_iter + 8) break;
                    }
                }
                if (rc) break;
                rn.go("accumulate", k_accumulate<R>, dim3(nb_e, n_out), dim3(TPB), N, so2, (const SysState*)sst,
                      (const cx<R>*)x, (long long)N, job.x64);
            } else {
                // one GMRES(m) cycle on the scaled residual
                const long long ldV = (long long)(mres + 1) * N;
                rn.go("inner_rhs", k_inner_rhs<R>, dim3(nb_e, n_in), dim3(TPB), N, si, (const SysState*)sst, res, V, ldV);
                rn.go("gmres_start", k_gmres_cycle_start, dim3(gs), dim3(128), nsys, mres, (const int*)inner, g);
                if (tune && mdl->mv_variant[sizeof(R) == 4 ? 0 : 1] < 0) {
                    if (int trc = tune_matvec<R>(rn, mdl, (const int*)sys_e, si, n_in, (const cx<R>*)diagR, (const cx<R>*)V, ldV,
                                                 w, (long long)N, (const double2*)nullptr, partA, 0)) {
                        fail(trc);
                        break;
                    }
                }
                const int mvv = mdl->mv_variant[sizeof(R) == 4 ? 0 : 1];
                const Sel sc_out{olist, nullptr};  // systems that run this cycle (for the final combination)
                for (int j = 0; j < mres; ++j) {
                    const Sel sc{ilist, inner};
                    const cx<R>* vj = V + (long long)j * N;
                    if (pspan < 0) {
                        launch_matvec<R, M>(rn, "matvec", md, (const int*)sys_e, sc, n_in, (const cx<R>*)diagR, vj, ldV, w,
                                            (long long)N, (const double2*)nullptr, partA, 0, mvv);
                    } else {
                        precond(sc, n_in, vj, ldV, z, N, nullptr);
                        launch_matvec<R, M>(rn, "matvec", md, (const int*)sys_e, sc, n_in, (const cx<R>*)diagR,
                                            (const cx<R>*)z, (long long)N, w, (long long)N, (const double2*)nullptr, partA, 0,
                                            mvv);
                    }
                    rn.go("gmres_dots", k_vdots<R>, dim3(nb_v, n_in), dim3(TPB), N, mres, sc, (const cx<R>*)V, j,
                          (const cx<R>*)w, partA);
                    rn.go("gmres_hreduce", k_hreduce, dim3(cdiv_u(j + 1, HR_K), nsys), dim3(HR_K, HR_G), nsys, mres,
                          (const int*)inner, j, (const double2*)partA, nb_v, h1);
                    rn.go("gmres_update_dots", k_vupdate<R>, dim3(nb_v, n_in), dim3(TPB), N, mres, sc, (const cx<R>*)V, j,
                          (const double2*)h1, w, 0, partA);
                    rn.go("gmres_hreduce", k_hreduce, dim3(cdiv_u(j + 1, HR_K), nsys), dim3(HR_K, HR_G), nsys, mres,
                          (const int*)inner, j, (const double2*)partA, nb_v, h2);
                    rn.go("gmres_update_norm", k_vupdate<R>, dim3(nb_v, n_in), dim3(TPB), N, mres, sc, (const cx<R>*)V, j,
                          (const double2*)h2, w, 1, partB);
                    cudaMemsetAsync(cnt, 0, sizeof(int), st);
                    cudaMemsetAsync(ilist, 0xff, nsys * sizeof(int), st);
                    rn.go("gmres_givens", k_givens, dim3(cdiv_u(nsys, GV_W)), dim3(32 * GV_W), nsys, mres, sst, inner,
                          (const double2*)h1,
                          (const double2*)h2, (const double2*)partB, nb_v, H, cs, sn, g, invh, o.max_iter, cnt, ilist);
                    if (j + 1 < mres)
                        rn.go("gmres_scale", k_vscale<R>, dim3(nb_e, n_in), dim3(TPB), N, mres, sc, (const double*)invh,
                              (const SysState*)sst, (const cx<R>*)w, V);
                    if ((j + 1) % std::max(1, o.check_every) == 0 || j + 1 == mres) {
                        cudaMemcpyAsync(hcnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
                        if (cudaStreamSynchronize(st) != cudaSuccess) {
                            fail(vbk_cuda_fail(cudaGetLastError(), "GMRES iterations"));
                            break;
                        }
                        rn.flush();
                        if (hcnt[0] == 0) break;
                        n_in = (unsigned)hcnt[0];
                    }
                }
                if (rc) break;
                rn.go("gmres_trisolve", k_tri_solve, dim3(gs), dim3(128), nsys, mres, (const SysState*)sst, (const int*)outer,
                      (const double2*)H, (const double2*)g, yv);
                rn.go("gmres_combine", k_vcombine<R>, dim3(nb_e, n_out), dim3(TPB), N, mres, sc_out, (const SysState*)sst,
                      (const cx<R>*)V, (const double2*)yv, w);
                if (pspan < 0) {
                    rn.go("accumulate", k_accumulate<R>, dim3(nb_e, n_out), dim3(TPB), N, sc_out, (const SysState*)sst,
                          (const cx<R>*)w, (long long)N, job.x64);
                } else {
                    precond(sc_out, n_out, w, N, z, N, nullptr);
                    rn.go("accumulate", k_accumulate<R>, dim3(nb_e, n_out), dim3(TPB), N, sc_out, (const SysState*)sst,
                          (const cx<R>*)z, (long long)N, job.x64);
                }
            }
            if (cudaError_t ce = cudaGetLastError(); ce != cudaSuccess) {
                fail(vbk_cuda_fail(ce, "iteration kernels"));
                break;
            }
            if (rn.first_error != cudaSuccess) {
                fail(VBK_ERR_CUDA);
                break;
            }
        }
        if (rc) break;
        if (dfr && !cluster)
            rn.go("df_out", k_df_out, dim3(cdiv_u((long long)nsys * N, 2 * TPB)), dim3(TPB), (long long)nsys * N, (const float4*)xs,
                  job.x64);
        // results
        if (cudaMemcpyAsync(hst, sst, nsys * sizeof(SysState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            fail(vbk_cuda_fail(cudaGetLastError(), "result copy"));
            break;
        }
        rn.flush();
        if (vbk_stream_fault_take()) {  // a streaming matvec stopped waiting for its copies: results not valid
            vbk_set_error("streaming matvec: a wait for shared-memory copies ran past its limit");
            fail(VBK_ERR_CUDA);
            break;
        }
        std::vector<int> hfail(nE, 0);
        if (block || pspan == 0) {  // zero pivots of the block factors or of the point preconditioner
            cudaMemcpy(hfail.data(), pfail, nE * sizeof(int), cudaMemcpyDeviceToHost);
        }
        bool all_ok = true;
        for (int s = 0; s < nsys; ++s) {
            SysState& S = hst[s];
            int status = S.status;
            if (hfail[job.sys_e[s]] && status != VBK_SYS_CONVERGED) status = VBK_SYS_PIVOT;
            if (status != VBK_SYS_CONVERGED && status != VBK_SYS_ZERO_RHS) all_ok = false;
            if (stats) {
                stats[s].status = status;
                stats[s].iterations = S.iters;
                stats[s].refinements = S.refines;
                stats[s].rel_residual = S.bnorm > 0 ? S.rnorm / S.bnorm : 0.0;
            }
        }
        if (!all_ok) rc = VBK_ERR_NOT_CONVERGED;
    } while (0);
    cudaFreeAsync(wsbase, st);
    if (pbuf.mem) cudaFreeAsync(pbuf.mem, st);
    cudaStreamSynchronize(st);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (pgexec) cudaGraphExecDestroy(pgexec);
    return rc;
}

template <class R>
void block_precond(Runner& rn, const DevPlanBuf& pb, int N, Sel sel, unsigned ny, const int* sys_e, const cx<R>* F,
                   const SysState* sst, int upd, cx<R>* x, cx<R>* r, long long rs, const cx<R>* p, const cx<R>* q, cx<R>* z,
                   long long zs, double2* part_rr, double2* part_rz) {
    if (pb.staged) {
        const size_t smem = (size_t)pb.pd.L * (SG + 1) * sizeof(cx<R>);
        const dim3 g((pb.pd.nblk + SG - 1) / SG, ny);
        auto launch = [&](auto kern) {
            if (g.x == 0 || g.y == 0) return;
            rn.go_smem(upd ? "cocg_update_precond" : "block_apply", kern, g, dim3(STPB), smem, pb.pd, sel.list, sel.act, sys_e,
                       F, sst, upd, x, r, rs, p, q, z, zs, part_rr, part_rz);
        };
        switch (pb.P) {
            case 2: launch(k_block_staged<R, 2>); break;
            case 4: launch(k_block_staged<R, 4>); break;
            case 8: launch(k_block_staged<R, 8>); break;
            default: launch(k_block_staged<R, 16>); break;
        }
        return;
    }
    if (upd) {
        // generic path: the COCG update as its own kernel, then the block solve
        rn.go("cocg_update", k_cocg_update<R>, dim3(cdiv_u(N, TPB), ny), dim3(TPB), N, sel, sst, sys_e, 1,
              (const cx<R>*)nullptr, x, r, p, q, z, part_rr, (double2*)nullptr);
    }
    if (pb.wide) {
        if (ny == 0) return;
        rn.go("block_apply_wide", k_level_apply<R>, dim3(ny, pb.pd.nblk), dim3(4 * 32 * ((pb.pd.S + 31) / 32)), pb.pd, sys_e,
              sel, F, (const cx<R>*)r, rs, z, zs, part_rz);
        return;
    }
    rn.go("block_apply", k_block_apply<R>, dim3((pb.pd.nblk + BTPB - 1) / BTPB, ny), dim3(BTPB), pb.pd, sys_e, sel, F,
          (const cx<R>*)r, rs, z, zs, part_rz);
}

template <class R>
int dispatch(vbk_model* m, const SolveJob& job, const vbk_opts& o, vbk_stats* st, cudaStream_t s) {
    switch (m->M) {
        case 1: return Solver<R, 1>::run(m, job, o, st, s);
        case 2: return Solver<R, 2>::run(m, job, o, st, s);
        case 3: return Solver<R, 3>::run(m, job, o, st, s);
        case 4: return Solver<R, 4>::run(m, job, o, st, s);
    }
    vbk_set_error("unsupported number of modes");
    return VBK_ERR_UNSUPPORTED;
}

// ---------------------------------------------------------------- stand-alone operators
// y = A x (op = 0) or z = B^-1 r (op = 1) for n_E energies x nvec vectors, FP64 in and out.
template <class R, int M>
int operator_run(vbk_model* m, int op, int nE, const double* E, int nvec, int span, const double2* x, double2* y,
                 cudaStream_t st, int variant) {
    const int N = m->N;
    const bool mixed = sizeof(R) == 4;
    const long long nsys = (long long)nE * nvec;
    BlockPlan bp;
    DevPlanBuf pbuf;
    const bool block = op == 1 && span > 0;
    DevModel md = m->dm;  // own copy: the per-call buffers of q-dependent couplings are set below
    const bool sand = md.nsc > 0;
    if (block) {
        int rc = vbk_make_block_plan(m, span, &bp);
        if (rc) return rc;
        rc = upload_plan(bp, m, st, &pbuf);
        if (!rc) rc = prepare_staged<R>(pbuf);
        if (rc) {
            if (pbuf.mem) cudaFreeAsync(pbuf.mem, st);
            return rc;
        }
    }
    if (op == 0) {
        if (variant >= MV_NVAR || (variant >= 0 && !mv_valid(m->dm, variant, sizeof(cx<R>)))) {
            vbk_set_error("matvec variant not available for this model and precision");
            return VBK_ERR_INVALID_ARG;
        }
        if (int rc = prepare_matvec<R>(m->dm)) return rc;
    }
    size_t bytes = carve_size<double2>((size_t)nE * N) + carve_size<float2>(mixed ? (size_t)nE * N : 1) +
                   2 * carve_size<cx<R>>(mixed ? (size_t)nsys * N : 1) + carve_size<int>(nsys) + carve_size<double>(nE) +
                   carve_size<int>(nE) + (block ? carve_size<cx<R>>((size_t)nE * factor_entries(bp, N)) : 0);
    const size_t n_g = sand ? (size_t)nE * md.npair * md.Nnu : 1, n_w = sand ? (size_t)nsys * md.nsc * md.Nnu : 1;
    if (sand)
        bytes += carve_size<double2>(n_g) + carve_size<float2>(n_g) + carve_size<double2>((size_t)nE * N) +
                 carve_size<float2>((size_t)nE * N) + carve_size<double2>(n_w);
    char* base = nullptr;
    if (vbk_alloc(m, (void**)&base, bytes, st) != cudaSuccess) {
        if (pbuf.mem) cudaFreeAsync(pbuf.mem, st);
        cudaGetLastError();
        vbk_set_error("operator workspace allocation failed");
        return VBK_ERR_OOM;
    }
    char* p = base;
    double2* d64 = carve<double2>(p, (size_t)nE * N);
    float2* d32 = carve<float2>(p, mixed ? (size_t)nE * N : 1);
    cx<R>* xr = carve<cx<R>>(p, mixed ? (size_t)nsys * N : 1);
    cx<R>* yr = carve<cx<R>>(p, mixed ? (size_t)nsys * N : 1);
    int* se = carve<int>(p, nsys);
    double* dE = carve<double>(p, nE);
    int* pfail = carve<int>(p, nE);
    cx<R>* F = block ? carve<cx<R>>(p, (size_t)nE * factor_entries(bp, N)) : nullptr;
    if (sand) {
        md.sg64 = carve<double2>(p, n_g);
        md.sg32 = mixed ? carve<float2>(p, n_g) : nullptr;
        md.sfd64 = carve<double2>(p, (size_t)nE * N);
        md.sfd32 = mixed ? carve<float2>(p, (size_t)nE * N) : nullptr;
        md.sw64 = carve<double2>(p, n_w);
        md.sw32 = reinterpret_cast<float2*>(md.sw64);
    }
    if (!mixed) {
        xr = reinterpret_cast<cx<R>*>(const_cast<double2*>(x));
        yr = reinterpret_cast<cx<R>*>(y);
    }
    const cx<R>* diagR = mixed ? reinterpret_cast<const cx<R>*>(d32) : reinterpret_cast<const cx<R>*>(d64);
    std::vector<int> hse(nsys);
    for (long long s = 0; s < nsys; ++s) hse[s] = (int)(s / nvec);
    int rc = VBK_OK;
    Runner rn{m, st, m->op_timing != 0, {}, {}};
    const Sel none{nullptr, nullptr};
    if (cudaMemcpyAsync(se, hse.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dE, E, nE * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(pfail, 0, nE * sizeof(int), st) != cudaSuccess) {
        rc = vbk_cuda_fail(cudaGetLastError(), "operator set-up");
    } else {
        if (sand) rn.go("sandwich_table", k_sand_table, dim3(cdiv_u(md.Nnu, TPB), nE), dim3(TPB), md, nE, (const double*)dE);
        rn.go("diag_table", k_diag_table<M>, dim3(cdiv_u(N, TPB), nE), dim3(TPB), md, nE, (const double*)dE, d64,
              mixed ? d32 : (float2*)nullptr, (float2*)nullptr, (float4*)nullptr, (int*)nullptr);
        const dim3 ge(cdiv_u(N, TPB), (unsigned)nsys);
        if (mixed) rn.go("narrow", k_inner_rhs_plain, dim3(cdiv_u(nsys * N, TPB)), dim3(TPB), nsys * N, x, reinterpret_cast<float2*>(xr));
        if (op == 0) {
            launch_matvec<R, M>(rn, "matvec", md, (const int*)se, none, (unsigned)nsys, diagR, (const cx<R>*)xr, (long long)N,
                                yr, (long long)N, (const double2*)nullptr, (double2*)nullptr, 0,
                                variant >= 0 ? variant : m->mv_variant[sizeof(R) == 4 ? 0 : 1]);
        } else if (block) {
            factor_blocks<R, M>(rn, md, pbuf, nE, diagR, F, pfail);
            block_precond<R>(rn, pbuf, N, none, (unsigned)nsys, (const int*)se, (const cx<R>*)F, (const SysState*)nullptr, 0,
                             nullptr, xr, (long long)N, nullptr, nullptr, yr, (long long)N, nullptr, nullptr);
        } else {
            rn.go("point_precond", k_point_precond<R>, ge, dim3(TPB), N, (const int*)se, none, span < 0 ? -1 : 0,
                  diagR, (const cx<R>*)xr, (long long)N, yr, (long long)N, (double2*)nullptr);
        }
        if (mixed) rn.go("widen", k_widen, dim3(cdiv_u(nsys * N, TPB)), dim3(TPB), nsys * N, (const float2*)reinterpret_cast<float2*>(yr), y);
        if (cudaError_t ce = cudaGetLastError(); ce != cudaSuccess) rc = vbk_cuda_fail(ce, "operator kernels");
        if (!rc && rn.first_error != cudaSuccess) rc = VBK_ERR_CUDA;
        if (!rc && block) {
            std::vector<int> hf(nE);
            if (cudaMemcpyAsync(hf.data(), pfail, nE * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = vbk_cuda_fail(cudaGetLastError(), "operator pivot check");
            } else {
                for (int e = 0; e < nE; ++e)
                    if (hf[e]) {
                        vbk_set_error("zero pivot in the L D L^T factor of a preconditioner block");
                        rc = VBK_ERR_NOT_CONVERGED;
                    }
            }
        }
    }
    if (rn.timing) {  // per-kernel timings of this call (vbk_set_op_timing)
        if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = vbk_cuda_fail(cudaGetLastError(), "operator timing");
        rn.flush();
        if (vbk_stream_fault_take() && !rc) {
            vbk_set_error("streaming matvec: a wait for shared-memory copies ran past its limit");
            rc = VBK_ERR_CUDA;
        }
    }
    cudaFreeAsync(base, st);
    if (pbuf.mem) cudaFreeAsync(pbuf.mem, st);
    return rc;
}

template <class R>
int operator_dispatch(vbk_model* m, int op, int nE, const double* E, int nvec, int span, const double2* x, double2* y,
                      cudaStream_t st, int variant) {
    switch (m->M) {
        case 1: return operator_run<R, 1>(m, op, nE, E, nvec, span, x, y, st, variant);
        case 2: return operator_run<R, 2>(m, op, nE, E, nvec, span, x, y, st, variant);
        case 3: return operator_run<R, 3>(m, op, nE, E, nvec, span, x, y, st, variant);
        case 4: return operator_run<R, 4>(m, op, nE, E, nvec, span, x, y, st, variant);
    }
    vbk_set_error("unsupported number of modes");
    return VBK_ERR_UNSUPPORTED;
}

}  // namespace

int vbk_solve_job(vbk_model* m, const SolveJob& job, const vbk_opts& o, vbk_stats* st, cudaStream_t s) {
    m->timers.clear();
    m->launches = 0;
    if (o.precision == VBK_MIXED) return dispatch<float>(m, job, o, st, s);
    return dispatch<double>(m, job, o, st, s);
}

int vbk_operator_run(vbk_model* m, int op, int nE, const double* E, int nvec, int span, const double2* x, double2* y,
                     int precision, cudaStream_t st, int variant) {
    if (m->op_timing) {
        m->timers.clear();
        m->launches = 0;
    }
    if (precision == VBK_MIXED) return operator_dispatch<float>(m, op, nE, E, nvec, span, x, y, st, variant);
    return operator_dispatch<double>(m, op, nE, E, nvec, span, x, y, st, variant);
}

// =========================================================== allocation-free operator apply
// Some callers cannot allocate device memory when they apply the operator: a process whose
// device memory another framework's allocator has already reserved almost entirely, or a
// real-time loop that forbids allocation after start-up.  vbk_matvec_noalloc serves them: it
// applies A(E) in FP64 like vbk_matvec, but keeps its scratch (the energies, the system-to-
// energy map and the diagonal tables) in the fixed device array below instead of allocating.
// The array is part of the library image, so every GPU that loads the library holds it until
// the process exits.  Every call reuses it and it keeps the last call's contents; everything a
// call reads is written by that call first.  Two calls that overlap on the GPU (on different
// streams, or from different host threads) race on it.
#define VBK_NOALLOC_SCRATCH_BYTES (8u << 20)  // 8 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[VBK_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr int NOALLOC_MAX_VECS = 4096;  // vectors (n_E * n_vec) per call
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array for the current device, looked up once per device with
// that device current.  Host code must not pass &g_noalloc_scratch to a kernel: on the host that
// name is only a stand-in for the device symbol.
int noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return vbk_cuda_fail(ce, "noalloc: current device");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        vbk_set_error("noalloc: device index beyond the supported range");
        return VBK_ERR_UNSUPPORTED;
    }
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (ce != cudaSuccess || !p) return vbk_cuda_fail(ce, "noalloc: scratch symbol address");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return VBK_OK;
}

template <int M>
int noalloc_run(vbk_model* m, int nE, const double* E, int nvec, const double2* x, double2* y, cudaStream_t st) {
    const int N = m->N;
    const long long nsys = (long long)nE * nvec;
    // the host-side system map below holds at most NOALLOC_MAX_VECS entries
    if (nsys > NOALLOC_MAX_VECS) {
        vbk_set_error("noalloc: n_E * n_vec = " + std::to_string(nsys) + " vectors exceed the limit of " +
                      std::to_string(NOALLOC_MAX_VECS) + " per call; use vbk_matvec or split the batch");
        return VBK_ERR_INVALID_ARG;
    }
    // scratch layout: E [nE] | sys_e [nsys] | diag [nE][N]
    const size_t off_se = ((size_t)nE * sizeof(double) + 255) & ~size_t(255);
    const size_t off_dg = (off_se + (size_t)nsys * sizeof(int) + 255) & ~size_t(255);
    const size_t need = off_dg + (size_t)nE * N * sizeof(double2);
    if (need > VBK_NOALLOC_SCRATCH_BYTES) {
        vbk_set_error("noalloc: n_E * N complex entries (plus energies and the system map) exceed the " +
                      std::to_string(VBK_NOALLOC_SCRATCH_BYTES) + "-byte scratch array (need " + std::to_string(need) +
                      " bytes); use vbk_matvec or fewer energies per call");
        return VBK_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    if (int rc = noalloc_scratch(&base)) return rc;
    char* sb = (char*)base;
    double* dE = (double*)sb;
    int* se = (int*)(sb + off_se);
    double2* d64 = (double2*)(sb + off_dg);
    int hse[NOALLOC_MAX_VECS];
    for (long long s = 0; s < nsys; ++s) hse[s] = (int)(s / nvec);
    cudaError_t ce;
    if ((ce = cudaMemcpyAsync(dE, E, nE * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (ce = cudaMemcpyAsync(se, hse, nsys * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return vbk_cuda_fail(ce, "noalloc: copies into scratch");
    Runner rn{m, st, false, {}, {}};
    rn.go("diag_table", k_diag_table<M>, dim3(cdiv_u(N, TPB), nE), dim3(TPB), m->dm, nE, (const double*)dE, d64,
          (float2*)nullptr, (float2*)nullptr, (float4*)nullptr, (int*)nullptr);
    const Sel none{nullptr, nullptr};
    launch_matvec_v<double>(rn, 9, "matvec_fp64", m->dm, (const int*)se, none, (unsigned)nsys, (const double2*)d64, x,
                            (long long)N, y, (long long)N, (const double2*)nullptr, (double2*)nullptr, 0);
    if ((ce = cudaGetLastError()) != cudaSuccess) return vbk_cuda_fail(ce, "noalloc: kernels");
    if (rn.first_error != cudaSuccess) return VBK_ERR_CUDA;
    // the host-side system map must outlive its copy
    if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return vbk_cuda_fail(ce, "noalloc: completion");
    return VBK_OK;
}

}  // namespace

extern "C" int vbk_matvec_noalloc(vbk_model* m, int n_E, const double* E, int n_vec, const void* x_dev, void* y_dev,
                                  void* stream) {
    vbk_set_error("");
    if (!m) {
        vbk_set_error("model handle is NULL");
        return VBK_ERR_INVALID_ARG;
    }
    if (n_E < 1 || n_vec < 1 || !E || !x_dev || !y_dev) {
        vbk_set_error("noalloc: sizes and buffers must be given");
        return VBK_ERR_INVALID_ARG;
    }
    for (int k = 0; k < n_E; ++k)
        if (!std::isfinite(E[k])) {
            vbk_set_error("energies must be finite");
            return VBK_ERR_INVALID_ARG;
        }
    if (m->dm.nsc) {
        vbk_set_error("noalloc: q-dependent continuum couplings need per-call tables beyond the scratch array; use vbk_matvec");
        return VBK_ERR_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const double2* x = (const double2*)x_dev;
    double2* y = (double2*)y_dev;
    switch (m->M) {
        case 1: return noalloc_run<1>(m, n_E, E, n_vec, x, y, st);
        case 2: return noalloc_run<2>(m, n_E, E, n_vec, x, y, st);
        case 3: return noalloc_run<3>(m, n_E, E, n_vec, x, y, st);
        case 4: return noalloc_run<4>(m, n_E, E, n_vec, x, y, st);
    }
    vbk_set_error("unsupported number of modes");
    return VBK_ERR_UNSUPPORTED;
}
