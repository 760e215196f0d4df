// Streaming batched matvec y = A(E) x (Sec. III matrix-free product, Eq. U) for models whose
// rows of mode 0 are short (n_s * N_nu / n_0 <= 640 elements, every stencil point involving at
// most two modes).
//
// The operator is a stencil over the product basis: y(d, nu) = diag(E)(d, nu) x(d, nu) +
// sum_k c_k(nu) x(dp_k, nu + lin_k), and every coefficient c_k(nu) is a product of one factor
// that depends on the index of mode 0 only and one that depends on the other modes only (the
// primary-mode row of the point, times the oscillator table of its secondary mode).  A "row" is
// the set of elements of one state with a fixed index n_0 (R = N_nu / n_0 contiguous entries).
//
// Persistent CTAs walk tiles (S systems, a strip of TR rows of every state).  A tile needs, per
// system and state plane, the contiguous window of x that its rows reach (the strip widened by
// the smallest and largest in-plane offset) and the strip's rows of the diagonal table.  A
// producer warp issues them as bulk asynchronous copies (cp.async.bulk, the TMA engine's untiled
// form) into a ring of shared-memory stages, each stage with a "full" mbarrier that counts the
// bytes in and an "empty" one the consumer warps arrive on when they are done with it; while
// the consumers compute tile i, the copies of the next tiles are in flight.  Each consumer
// thread owns one (state, in-row position) and TR / RG rows of a tile: its factors of the
// in-row modes stay in registers for the whole launch, the factors of mode 0 come from a table
// in shared memory (one broadcast load per point and row), and every neighbour is read from the
// staged window.  y leaves by coalesced stores straight from registers.
//
// DRAM traffic per tile: the windows (the halo rows are re-read from L2 by the neighbouring
// strip's CTA, which runs at the same time), the diagonal rows (once for the systems of the
// tile that share an energy), and y.
#include <algorithm>

#include "vbk_internal.cuh"
#include "vbk_device.cuh"

// Set by a CTA whose wait for its own copies ran past the poll limit; the kernel then carries on
// (its output is not valid) rather than wait without end.  The byte counts are exact, so this is
// not expected; the host reads and clears it with vbk_stream_fault_take().
__device__ unsigned int g_vbk_stream_fault = 0;

namespace {

constexpr int ST_NPM = 16;                          // stencil points per state (padded with zero points)
constexpr int ST_MAXT = 640;                        // consumer threads per CTA at most (and one producer warp)
constexpr int ST_SMALLT = 352;                      // blocks of at most this many threads: two per SM
constexpr size_t ST_SMEM_MAX = 220 * 1024;          // dynamic shared memory of a CTA at most
constexpr unsigned long long ST_WAIT_NS = 1000000000ull;  // a stage barrier wait gives up after 1 s

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// one arrival (the barrier's whole count) that also announces `bytes` of copies to come
__device__ __forceinline__ void mbar_arrive_expect(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// true once the phase of parity `parity` has completed; the thread may be suspended (up to a
// millisecond) while it waits, so waiting warps take no issue slots from the working ones
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long st_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16), completion
// counted on `bar`
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// coefficient type: a packed pair (c, c) in FP32 (one FP32x2 FMA per complex update), c in FP64
template <class R> struct StCoef;
template <> struct StCoef<float> { typedef float2 T; };
template <> struct StCoef<double> { typedef double T; };
__device__ __forceinline__ float2 st_pack(float v) { return make_float2(v, v); }
__device__ __forceinline__ double st_pack(double v) { return v; }
__device__ __forceinline__ float2 st_mul(float2 a, float2 b) { return fmul2(a, b); }
__device__ __forceinline__ double st_mul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 st_fma(float2 c, float2 v, float2 acc) { return ffma2(c, v, acc); }
__device__ __forceinline__ double2 st_fma(double c, double2 v, double2 acc) {
    return make_double2(fma(c, v.x, acc.x), fma(c, v.y, acc.y));
}
// entry n of the primary-mode coefficient rows (-coef (q^k)_{n, n + delta})
template <class R> __device__ __forceinline__ R row_val(const DevModel& md, int n);
template <> __device__ __forceinline__ float row_val<float>(const DevModel& md, int n) { return md.rct[n].x; }
template <> __device__ __forceinline__ double row_val<double>(const DevModel& md, int n) { return md.rct64[n]; }
template <class R> __device__ __forceinline__ const R* st_tab(const DevModel& md);
template <> __device__ __forceinline__ const float* st_tab<float>(const DevModel& md) { return md.tab32; }
template <> __device__ __forceinline__ const double* st_tab<double>(const DevModel& md) { return md.tab64; }

// primary mode of point q of state d (the points of a state are grouped by primary mode)
__device__ __forceinline__ int st_primary(const DevModel& md, int d, int q) {
    int m = 0, end = md.rcnt[d][0];
    while (q >= end && m < MAXM - 1) end += md.rcnt[d][++m];
    return m;
}
template <class R> __device__ __forceinline__ cx<R> st_warp_sum(cx<R> v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ int st_sel(const int (&n)[MAXM], int m) {
    int r = n[0];
#pragma unroll
    for (int k = 1; k < MAXM; ++k) r = (m == k) ? n[k] : r;
    return r;
}

// Wait for the phase of parity `par` of the barrier at `bar`; gives up after ST_WAIT_NS, records
// that in g_vbk_stream_fault and returns false (the data it guards are then not valid).
__device__ __forceinline__ bool st_wait(unsigned bar, unsigned par) {
    if (mbar_try_wait(bar, par)) return true;
    const unsigned long long t0 = st_clock_ns();
    while (!mbar_try_wait(bar, par))
        if (st_clock_ns() - t0 > ST_WAIT_NS) {
            atomicOr(&g_vbk_stream_fault, 1u);
            return false;
        }
    return true;
}
// barrier over the consumer warps only (named barrier 1; the producer warp is not part of it)
__device__ __forceinline__ void st_cons_sync(int ncons) { asm volatile("bar.sync 1, %0;" ::"r"(ncons) : "memory"); }

// The S systems' entries of one window slot (the systems' windows lie `sysb` bytes apart).
template <class R, int S>
__device__ __forceinline__ void st_load_sys(const unsigned char* p, int sysb, cx<R> (&v)[S]) {
#pragma unroll
    for (int k = 0; k < S; ++k) v[k] = *reinterpret_cast<const cx<R>*>(p + k * sysb);
}

// Systems of tile t: list entries [g S, g S + S) of strip si (-1: no system / retired).
template <int S>
__device__ __forceinline__ void st_tile(const StreamPlan& p, int t, int nlist, const int* list, const int* act, int (&sy)[S],
                                        int& si) {
    const int g = t / p.nstrip;
    si = t - g * p.nstrip;
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const int li = g * S + k;
        int s = -1;
        if (li < nlist) {
            s = list ? list[li] : li;
            if (s >= 0 && act && !act[s]) s = -1;
        }
        sy[k] = s;
    }
}

// NPG: stencil points per state (padded with zero points); PLAIN: y = A x with no residual form
// and no partial sums (b == null, red == 0); MAXT, MINB: launch bounds.
template <class R, int S, int NPG, bool PLAIN, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_matvec_stream(DevModel md, StreamPlan p, const int* __restrict__ sys_e,
                                                             const int* __restrict__ list, const int* __restrict__ act,
                                                             int nlist, const cx<R>* __restrict__ diag,
                                                             const cx<R>* __restrict__ x, long long xs,
                                                             cx<R>* __restrict__ y, long long ys,
                                                             const double2* __restrict__ b, double2* __restrict__ part,
                                                             int red) {
    using C = cx<R>;
    using CR = typename StCoef<R>::T;
    using CR2 = typename std::conditional<sizeof(R) == 4, float4, double2>::type;  // two table entries
    constexpr int NPT = NPG;    // table columns per (state, row)
    constexpr int NPROD = 32;   // one producer warp
    static_assert(NPT % 2 == 0, "table rows are read in pairs");
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) unsigned long long fullb[ST_MAXSTAGE], emptyb[ST_MAXSTAGE];
    __shared__ int info[ST_MAXSTAGE][3 * S + 1];  // per stage: systems, diagonal buffer (-1: global), energies, strip
    __shared__ C redsh[32][S];
    const int tid = threadIdx.x, ns = md.ns, Nnu = md.Nnu, N = md.N, nb0 = md.nb[0];
    const int Rl = p.R, plane = ns * Rl;
    const int ncons = (int)blockDim.x - NPROD;  // consumer threads: the warps after the producers
    const int ct = tid - NPROD;
    const bool live = ct >= 0 && ct < p.RG * plane;
    const int rg = live ? ct / plane : 0;
    const int rem = live ? ct - rg * plane : 0;
    const int d = rem / Rl, col = rem - d * Rl;
    CR* cgt = reinterpret_cast<CR*>(sm + (size_t)p.nst * p.stage_bytes);  // [ns][nb0][NPT] factors of mode 0
    const R* tab = st_tab<R>(md);
    // bytes between one window slot and the next, and between two systems' windows
    constexpr int slotb = (int)sizeof(C);
    const int sysb = ns * p.W * (int)sizeof(C);

    // this thread's factors of the in-row modes (table column order) and the byte offsets of the
    // stencil points within the windows
    CR cu[NPT];
    int off[NPG];
#pragma unroll
    for (int q = 0; q < NPT; ++q) cu[q] = st_pack((R)0);
#pragma unroll
    for (int q = 0; q < NPG; ++q) off[q] = 0;
    if (live) {
        int n[MAXM];
#pragma unroll
        for (int m = 0; m < MAXM; ++m) n[m] = (m >= 1 && m < md.M) ? (col / md.stride[m]) % md.nb[m] : 0;
        const int kb = md.rbeg[d], cnt = md.rbeg[d + 1] - kb;
        for (int q = 0; q < cnt && q < NPG; ++q) {
            const int m1 = st_primary(md, d, q);
            const int4 w = md.wdesc[kb + q];
            const int m2 = w.w & 0xff, dp = w.w >> 8;
            R v = (R)1;
            if (m1 >= 1) v *= row_val<R>(md, w.x / 8 + st_sel(n, m1));
            if (w.z >= 0 && m2 >= 1) v *= tab[w.z + st_sel(n, m2)];
#pragma unroll
            for (int j = 0; j < NPG; ++j)
                if (j == q) {
                    cu[j] = st_pack(v);
                    off[j] = ((dp - d) * p.W + w.y) * slotb;
                }
        }
    }
    // factors of mode 0 for every (state, row, point)
    for (int i = tid; i < ns * nb0 * NPT; i += blockDim.x) {
        const int dd = i / (nb0 * NPT), r2 = i - dd * nb0 * NPT, g = r2 / NPT, q = r2 - g * NPT;
        const int kb = md.rbeg[dd], cnt = md.rbeg[dd + 1] - kb;
        R v = (R)0;
        if (q < cnt) {
            const int m1 = st_primary(md, dd, q);
            const int4 w = md.wdesc[kb + q];
            v = (R)1;
            if (m1 == 0) v *= row_val<R>(md, w.x / 8 + g);
            if (w.z >= 0 && (w.w & 0xff) == 0) v *= tab[w.z + g];
        }
        cgt[i] = st_pack(v);
    }
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(sm);
    const unsigned fbase = (unsigned)__cvta_generic_to_shared(fullb);
    const unsigned ebase = (unsigned)__cvta_generic_to_shared(emptyb);
    const int ntile = ((nlist + S - 1) / S) * p.nstrip;
    const int G = gridDim.x;
    const unsigned dbytes = (unsigned)(ns * p.TR * Rl * (int)sizeof(C));  // one diagonal buffer of a stage
    if (tid == 0) {
        for (int s = 0; s < p.nst; ++s) {
            mbar_init(fbase + 8u * s, 1);                    // the producer's arrival (plus the bytes)
            mbar_init(ebase + 8u * s, (unsigned)ncons / 32);  // one arrival per consumer warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();  // the only block-wide barrier: the producer warp leaves the loop below early

    if (tid < NPROD) {
        // ------------------------------------------------------------ producer warp
        const int lane = tid & 31;
        int it = 0;
        // the systems and energies of 32 tiles at a time, one tile per lane (their global loads
        // overlap instead of forming one dependent chain per tile)
        int bsy[S], bse[S], bsi = 0;
        for (;; ++it) {
            const int t = blockIdx.x + it * G;
            if (t >= ntile) break;
            const int s = it % p.nst, u = it / p.nst;
            if ((it & 31) == 0) {
                const int tl = t + lane * G;
#pragma unroll
                for (int k = 0; k < S; ++k) bsy[k] = -1;
                if (tl < ntile) st_tile<S>(p, tl, nlist, list, act, bsy, bsi);
#pragma unroll
                for (int k = 0; k < S; ++k) bse[k] = bsy[k] >= 0 ? sys_e[bsy[k]] : -1;
            }
            int sy[S], si;
            int se[S], slot[S], ea = -1, eb = -1, nact = 0;
#pragma unroll
            for (int k = 0; k < S; ++k) {
                sy[k] = __shfl_sync(0xffffffffu, bsy[k], it & 31);
                se[k] = __shfl_sync(0xffffffffu, bse[k], it & 31);
            }
            si = __shfl_sync(0xffffffffu, bsi, it & 31);
            // up to ndg energies of the tile get their diagonal rows staged
#pragma unroll
            for (int k = 0; k < S; ++k) {
                slot[k] = -1;
                if (se[k] < 0) continue;
                ++nact;
                if (ea < 0 || se[k] == ea) {
                    ea = se[k];
                    slot[k] = 0;
                } else if (p.ndg > 1 && (eb < 0 || se[k] == eb)) {
                    eb = se[k];
                    slot[k] = 1;
                }
            }
            if (u > 0) {
                st_wait(ebase + 8u * s, (unsigned)((u - 1) & 1));  // the consumers released the stage
                // and its previous copies have landed (always so, unless a consumer gave up waiting
                // for them): the barrier's next phase then counts only the copies issued below
                st_wait(fbase + 8u * s, (unsigned)((u - 1) & 1));
            }
            if (it == 0 && p.delay_ns && lane == 0) {
                // test hook (vbk_debug_stream_delay): hold the first copies back; a delay past the
                // wait limit makes the consumers' first wait run out.  Bounded by the delay.
                const unsigned long long t0 = st_clock_ns();
                while (st_clock_ns() - t0 < p.delay_ns) __nanosleep(100000);
            }
            __syncwarp();
            const int g0 = si * p.TR, tre = min(p.TR, nb0 - g0);
            const long long wst = (long long)g0 * Rl + p.lo;
            unsigned char* stg = sm + (size_t)s * p.stage_bytes;
            const unsigned st0 = sbase + (unsigned)s * p.stage_bytes;
            const unsigned bar = fbase + 8u * s;
            if (tid == 0) {
#pragma unroll
                for (int k = 0; k < S; ++k) {
                    info[s][k] = sy[k];
                    info[s][S + k] = slot[k];
                    info[s][2 * S + k] = se[k];
                }
                info[s][3 * S] = si;
            }
            {
                const long long a0 = wst > 0 ? wst : 0, a1 = min(wst + p.W, (long long)Nnu);
                if (wst < 0 || wst + p.W > Nnu) {
                    // window slots outside the basis: zero (their coefficients are zero; the
                    // slots must hold finite values)
                    const int f0 = (int)(a0 - wst), b0 = (int)(a1 - wst), nz = f0 + (p.W - b0);
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        if (sy[k] < 0) continue;
                        for (int dp = 0; dp < ns; ++dp) {
                            C* w = reinterpret_cast<C*>(stg) + (size_t)(k * ns + dp) * p.W;
                            for (int j = lane; j < nz; j += 32) w[j < f0 ? j : b0 + (j - f0)] = mkc<R>(0, 0);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    const unsigned wb = a1 > a0 ? (unsigned)((a1 - a0) * (long long)sizeof(C)) : 0u;
                    const unsigned db = (unsigned)(tre * Rl * (int)sizeof(C));
                    const unsigned total =
                        (unsigned)nact * ns * wb + (ea >= 0 ? ns * db : 0u) + (eb >= 0 ? ns * db : 0u);
                    // generic-proxy accesses of this stage (the consumers' reads, the zero fill)
                    // come before the copy engine writes it
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive_expect(bar, total);  // release: the zeros and info[s] are visible after the wait
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        if (sy[k] < 0 || wb == 0) continue;
                        for (int dp = 0; dp < ns; ++dp) {
                            const C* src = x + (long long)sy[k] * xs + (long long)dp * Nnu + a0;
                            const unsigned dst =
                                st0 + (unsigned)(((long long)(k * ns + dp) * p.W + (a0 - wst)) * (long long)sizeof(C));
                            bulk_g2s(dst, src, wb, bar);
                        }
                    }
                    for (int jd = 0; jd < 2; ++jd) {
                        const int e = jd == 0 ? ea : eb;
                        if (e < 0) continue;
                        for (int dp = 0; dp < ns; ++dp) {
                            const C* src = diag + (long long)e * N + (long long)dp * Nnu + (long long)g0 * Rl;
                            bulk_g2s(st0 + p.win_bytes + jd * dbytes + (unsigned)(dp * p.TR * Rl * (int)sizeof(C)), src,
                                     db, bar);
                        }
                    }
                }
            }
        }
        // stay until the copies of the last use of every stage have landed
        if (lane == 0)
            for (int s = 0; s < p.nst && s < it; ++s) {
                const int ulast = (it - 1 - s) / p.nst;
                st_wait(fbase + 8u * s, (unsigned)(ulast & 1));
            }
        return;
    }

    // ---------------------------------------------------------------- consumer warps
    const int cw = ct >> 5, clane = ct & 31;
    const int trt = p.TR / p.RG;  // rows of a tile per thread
    const int rowb = Rl * slotb;  // bytes between a slot and the same slot one row further
    for (int it = 0;; ++it) {
        const int t = blockIdx.x + it * G;
        if (t >= ntile) break;
        const int s = it % p.nst;
        // a wait that ran out leaves the stage's record and data unset: no system is written
        const bool landed = st_wait(fbase + 8u * s, (unsigned)((it / p.nst) & 1));
        int sy[S], slot[S], se[S];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            sy[k] = landed ? info[s][k] : -1;
            slot[k] = landed ? info[s][S + k] : -1;
            se[k] = landed ? info[s][2 * S + k] : -1;
        }
        const int si = landed ? info[s][3 * S] : 0;
        const int g0 = si * p.TR, tre = min(p.TR, nb0 - g0);
        const unsigned char* stg = sm + (size_t)s * p.stage_bytes;
        C loc[S];
#pragma unroll
        for (int k = 0; k < S; ++k) loc[k] = mkc<R>(0, 0);
        const int r0 = rg * trt, r1 = min(r0 + trt, tre);
        if (live && r0 < r1) {
            const unsigned char* dgs = stg + p.win_bytes + (size_t)d * p.TR * Rl * sizeof(C);
            const unsigned char* wself = stg + (size_t)(d * p.W + (r0 * Rl + col - p.lo)) * slotb;
            for (int r = r0; r < r1; ++r, wself += rowb) {
                const int el = r * Rl + col;
                const CR2* cg2 = reinterpret_cast<const CR2*>(cgt + ((size_t)d * nb0 + g0 + r) * NPT);
                const long long gi = (long long)d * Nnu + (long long)g0 * Rl + el;
                C xi[S], acc[S];
                st_load_sys<R, S>(wself, sysb, xi);
#pragma unroll
                for (int k = 0; k < S; ++k) {
                    C dg;
                    if (slot[k] >= 0) dg = *reinterpret_cast<const C*>(dgs + (size_t)slot[k] * dbytes + (size_t)el * sizeof(C));
                    else dg = se[k] >= 0 ? diag[(long long)se[k] * N + gi] : mkc<R>(0, 0);
                    acc[k] = cmul<R>(dg, xi[k]);
                }
                // point q: coefficient c_q = (mode-0 factor of the row) (in-row factor of the
                // thread); zero points (past a state's count) add 0 * x(self)
                auto apply = [&](int q, CR cq) {
                    C v[S];
                    st_load_sys<R, S>(wself + off[q], sysb, v);
#pragma unroll
                    for (int k = 0; k < S; ++k) acc[k] = st_fma(cq, v[k], acc[k]);
                };
#pragma unroll
                for (int j = 0; j < NPT / 2; ++j) {
                    const CR2 v = cg2[j];
                    if constexpr (sizeof(R) == 4) {
                        apply(2 * j, st_mul(make_float2(v.x, v.y), cu[2 * j]));
                        apply(2 * j + 1, st_mul(make_float2(v.z, v.w), cu[2 * j + 1]));
                    } else {
                        apply(2 * j, st_mul(v.x, cu[2 * j]));
                        apply(2 * j + 1, st_mul(v.y, cu[2 * j + 1]));
                    }
                }
#pragma unroll
                for (int k = 0; k < S; ++k) {
                    if (sy[k] < 0) continue;
                    C out = acc[k];
                    if (!PLAIN && b) {
                        const double2 bb = b[(long long)sy[k] * N + gi];
                        out = mkc<R>((R)bb.x - out.x, (R)bb.y - out.y);
                    }
                    y[(long long)sy[k] * ys + gi] = out;
                    if (PLAIN) continue;
                    if (red == 1) loc[k] = cfma<R>(xi[k], out, loc[k]);
                    else if (red == 2) {
                        const float ox = (float)out.x, oy = (float)out.y;  // norm for the stopping test: FP32 suffices
                        loc[k].x += (R)(ox * ox + oy * oy);
                    }
                }
            }
        }
        __syncwarp();
        if (clane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ebase + 8u * s) : "memory");
        if (!PLAIN && red) {
#pragma unroll
            for (int k = 0; k < S; ++k) {
                const C v = st_warp_sum<R>(loc[k]);
                if (clane == 0) redsh[cw][k] = v;
            }
            st_cons_sync(ncons);
#pragma unroll
            for (int k = 0; k < S; ++k)
                if (ct == k && sy[k] >= 0) {
                    C tot = mkc<R>(0, 0);
                    for (int q = 0; q < ncons / 32; ++q) tot = cadd<R>(tot, redsh[q][k]);
                    part[(long long)sy[k] * p.nstrip + si] = cvt_to_d<R>(tot);
                }
            st_cons_sync(ncons);  // redsh is free for the next tile
        }
    }
}

// instantiated shapes: S in {2, 4}, NPG in {8, 16}; each for up to 672 threads (one block per
// SM) or up to 352 threads (two blocks per SM)
template <class R, int S, int NPG, int MAXT, int MINB> void* st_kptr_p(bool plain) {
    return plain ? (void*)k_matvec_stream<R, S, NPG, true, MAXT, MINB> : (void*)k_matvec_stream<R, S, NPG, false, MAXT, MINB>;
}
template <class R, int S, int MAXT, int MINB> void* st_kptr_n(const StreamPlan& p, bool plain) {
    return p.npg == 8 ? st_kptr_p<R, S, 8, MAXT, MINB>(plain) : st_kptr_p<R, S, 16, MAXT, MINB>(plain);
}
template <class R, int MAXT, int MINB> void* st_kptr_t(const StreamPlan& p, bool plain) {
    return p.S == 4 ? st_kptr_n<R, 4, MAXT, MINB>(p, plain) : st_kptr_n<R, 2, MAXT, MINB>(p, plain);
}
template <class R> void* st_kernel_ptr(const StreamPlan& p, bool plain) {
    return p.threads <= ST_SMALLT ? st_kptr_t<R, ST_SMALLT, 2>(p, plain) : st_kptr_t<R, ST_MAXT + 32, 1>(p, plain);
}

int st_num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

// dynamic shared memory each kernel instance was opted in to, per device
constexpr int ST_NDEV = 16;
int st_optin[ST_NDEV][64] = {};
int st_kidx(bool fp32, const StreamPlan& p, bool plain) {
    const int shape = p.npg == 8 ? 0 : 1;
    return (p.threads <= ST_SMALLT ? 32 : 0) + (fp32 ? 0 : 16) + (p.S == 2 ? 0 : 8) + shape * 2 + (plain ? 1 : 0);
}

cudaError_t st_ensure_optin(bool fp32, const StreamPlan& p, bool plain) {
    int dev = 0;
    const size_t smem = p.smem;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= ST_NDEV) return cudaErrorInvalidDevice;
    int& cur = st_optin[dev][st_kidx(fp32, p, plain)];
    if ((int)smem <= cur) return cudaSuccess;
    void* kp = fp32 ? st_kernel_ptr<float>(p, plain) : st_kernel_ptr<double>(p, plain);
    const cudaError_t ce = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce == cudaSuccess) cur = (int)smem;
    return ce;
}

}  // namespace

// Tile shapes offered to the autotuner: (systems per tile, row groups, rows per tile, stages,
// diagonal buffers per stage).
static const int ST_CFG[][5] = {{4, 4, 8, 2, 2}, {4, 2, 4, 2, 2}, {2, 2, 8, 3, 1}, {2, 4, 16, 2, 1}};

int vbk_stream_nconfig() { return (int)(sizeof(ST_CFG) / sizeof(ST_CFG[0])); }

bool vbk_stream_plan(const DevModel& md, int cfg, size_t c, StreamPlan* out) {
    if (cfg < 0 || cfg >= vbk_stream_nconfig()) return false;
    if (md.nsc || !md.rok || md.M < 2 || md.ns < 1) return false;
    StreamPlan p;
    p.S = ST_CFG[cfg][0];
    const int nb0 = md.nb[0];
    p.R = md.Nnu / nb0;
    const int plane = md.ns * p.R;
    if (plane > ST_MAXT || p.R < 1) return false;
    int np = 0, lo = 0, hi = 0;
    for (int d = 0; d < md.ns; ++d) {
        np = std::max(np, md.rbeg[d + 1] - md.rbeg[d]);
        lo = std::min(lo, md.lmin[d]);
        hi = std::max(hi, md.lmax[d]);
    }
    if (np > ST_NPM) return false;
    p.npg = np <= 8 ? 8 : ST_NPM;
    p.np = p.npg;  // table columns per (state, row)
    if (c == 8) {  // 16-byte bulk copies of 8-byte entries: even offsets, sizes and row lengths
        if (p.R & 1) return false;
        lo = -((-lo + 1) & ~1);
        hi = (hi + 1) & ~1;
    }
    p.lo = lo;
    p.nst = ST_CFG[cfg][3];
    p.ndg = ST_CFG[cfg][4];
    const int rg = std::max(1, std::min(ST_CFG[cfg][1], ST_MAXT / plane));
    int tr = std::max(1, std::min(ST_CFG[cfg][2], nb0));
    for (;;) {
        p.RG = std::min(rg, tr);
        p.TR = (tr / p.RG) * p.RG;  // every thread takes TR / RG consecutive rows of a tile
        p.W = p.TR * p.R + (hi - lo);
        p.nstrip = (nb0 + p.TR - 1) / p.TR;
        p.win_bytes = (unsigned)((size_t)p.S * md.ns * p.W * c);
        // windows, then the diagonal buffers (the rows of up to ndg energies of the tile)
        p.stage_bytes = (unsigned)((p.win_bytes + (size_t)p.ndg * md.ns * p.TR * p.R * c + 127) & ~size_t(127));
        p.smem = (size_t)p.nst * p.stage_bytes + (size_t)md.ns * nb0 * p.np * 8;
        if (p.smem <= ST_SMEM_MAX || tr == 1) break;
        tr = (tr + 1) / 2;  // wide entries (FP64): shorter strips
    }
    p.threads = 32 + ((p.RG * plane + 31) / 32) * 32;  // a producer warp, then the consumer warps
    if (p.smem > ST_SMEM_MAX) return false;
    *out = p;
    return true;
}

// test hook: the next launch's producers hold their first copies back by this many milliseconds
static int g_stream_delay_ms = 0;

int vbk_debug_stream_delay_impl(int ms) {
    if (ms < 0 || ms > 10000) return VBK_ERR_INVALID_ARG;
    g_stream_delay_ms = ms;
    return VBK_OK;
}

cudaError_t vbk_stream_matvec(const DevModel& md, const StreamPlan& p_in, const int* sys_e, const int* list, const int* act,
                              int nlist, const void* diag, const void* x, long long xs, void* y, long long ys,
                              const double2* b, double2* part, int red, bool fp32, cudaStream_t st) {
    if (nlist <= 0) return cudaSuccess;
    StreamPlan p = p_in;
    p.delay_ns = (unsigned long long)g_stream_delay_ms * 1000000ull;
    g_stream_delay_ms = 0;  // one launch only
    const size_t c = fp32 ? 8 : 16;
    // bulk copies need 16-byte aligned sources: vector starts and the system strides
    if (((uintptr_t)x & 15) || ((uintptr_t)diag & 15) || ((xs * (long long)c) & 15)) return cudaErrorMisalignedAddress;
    // the opt-in is made outside any stream capture by vbk_stream_prepare (model preparation)
    const bool plain = b == nullptr && red == 0;
    cudaError_t ce = st_ensure_optin(fp32, p, plain);
    if (ce != cudaSuccess) return ce;
    void* kp = fp32 ? st_kernel_ptr<float>(p, plain) : st_kernel_ptr<double>(p, plain);
    int per_sm = 0;
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp, p.threads, p.smem);
    if (ce != cudaSuccess) return ce;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long ntile = (long long)((nlist + p.S - 1) / p.S) * p.nstrip;
    const int grid = (int)std::min<long long>(ntile, (long long)per_sm * st_num_sms());
    void* args[] = {(void*)&md, (void*)&p, (void*)&sys_e, (void*)&list, (void*)&act, (void*)&nlist, (void*)&diag,
                    (void*)&x, (void*)&xs, (void*)&y, (void*)&ys, (void*)&b, (void*)&part, (void*)&red};
    return cudaLaunchKernel(kp, dim3(grid), dim3(p.threads), args, p.smem, st);
}

int vbk_stream_prepare(const DevModel& md, bool fp32) {
    for (int cfg = 0; cfg < vbk_stream_nconfig(); ++cfg) {
        StreamPlan p;
        if (!vbk_stream_plan(md, cfg, fp32 ? 8 : 16, &p)) continue;
        for (int plain = 0; plain < 2; ++plain)
            if (const cudaError_t ce = st_ensure_optin(fp32, p, plain != 0); ce != cudaSuccess)
                return vbk_cuda_fail(ce, "streaming matvec shared-memory opt-in");
    }
    return VBK_OK;
}

unsigned vbk_stream_fault_take() {
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_vbk_stream_fault, sizeof(v)) != cudaSuccess) return 0;
    if (v) cudaMemcpyToSymbol(g_vbk_stream_fault, &z, sizeof(z));
    return v;
}
