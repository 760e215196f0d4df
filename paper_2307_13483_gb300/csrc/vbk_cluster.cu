// Fused mixed-precision solve on thread-block clusters (sm_103a).
//
// One cluster of n_s CTAs solves one system (E, v_i, mu) from start to finish: CTA d owns the
// N_nu unknowns of discrete state d.  Everything an FP32 COCG iteration touches lives on chip:
// the search direction p (with a zero halo), q = A p (then z = B^-1 r), the FP32 diagonal of
// A(E) and the inner correction in shared memory, the recursive residual in registers.  Stencil
// points that couple two states read the other CTA's p through distributed shared memory, and
// the bilinear forms p^T q, r^T z, ||r||^2 are summed per CTA and exchanged across the cluster,
// every CTA adding the n_s partials in rank order (so every CTA takes the same decisions).  The
// refinement (Sec. III stopping rule) runs in the same kernel: the residual b - A x in
// double-float arithmetic with x staged in shared memory (the same cluster exchange for the
// neighbours in other states), its norm, the convergence / stall / cap checks, the scaled inner
// right-hand side, and at the end psi = hi + lo in FP64.  Clusters take systems from a counter
// (highest index first: the higher energies of an ascending grid open more channels and take
// longer), so one launch solves the whole batch.
#include "vbk_internal.cuh"
#include "vbk_device.cuh"

namespace {

constexpr int CT = 512;       // threads per CTA (128 registers each: the residual stays in registers)
constexpr int CL_MAXPTS = 64;  // stencil points of one state

__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster; orders this CTA's shared-memory writes before the
// other CTAs' later reads (release / acquire)
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cl_map(unsigned local_addr, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
    return r;
}
// Loads from another CTA's shared memory.  Volatile keeps them in order with the cluster
// barriers (also volatile asm); without a memory clobber the compiler still schedules the
// ordinary shared-memory loads around them.
__device__ __forceinline__ float2 dsm_f2(unsigned a) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float4 dsm_f4(unsigned a) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ double dsm_d(unsigned a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ int dsm_i(unsigned a) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ unsigned sh_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// z = r / g in FP32 (the point preconditioner)
__device__ __forceinline__ float2 cdiv_f(float2 r, float2 g) {
    const float inv = __frcp_rn(g.x * g.x + g.y * g.y);
    return make_float2((r.x * g.x + r.y * g.y) * inv, (r.y * g.x - r.x * g.y) * inv);
}

// Shared-memory layout of the kernel (identical in every CTA of a launch, so that one CTA can
// address another's arrays): P [Nc + 2H] float2 | Q, DG, X [Nc] float2 each | rows (FP32
// pairs) | rows (double-float) | descriptors (FP32 pass, residual pass) | exchange slots.  The
// split solution XS [Nc + 2H] float4 overlays P, Q and part of DG during the residual.
struct ClLayout {
    int Nc, H, nrow, npt;
    size_t oQ, oDG, oX, oR32, oRD, oD1, oD2, oXch, bytes;
};
__host__ __device__ inline ClLayout cl_layout(int Nc, int H, int nrow, int npt) {
    ClLayout L;
    L.Nc = Nc;
    L.H = H;
    L.nrow = nrow;
    L.npt = npt;
    const size_t p = (size_t)(Nc + 2 * H) * 8;
    L.oQ = p;
    L.oDG = L.oQ + (size_t)Nc * 8;
    L.oX = L.oDG + (size_t)Nc * 8;
    L.oR32 = L.oX + (size_t)Nc * 8;
    L.oRD = L.oR32 + (size_t)nrow * 8;
    L.oD1 = (L.oRD + (size_t)nrow * 8 + 15) & ~size_t(15);
    L.oD2 = L.oD1 + (size_t)npt * 16;
    L.oXch = L.oD2 + (size_t)npt * 16;
    L.bytes = L.oXch + 2 * 4 * sizeof(double) + 16;  // two slots of four values, the system index
    return L;
}

template <int M, int EPT>
__global__ void __launch_bounds__(CT, 1) k_solve_cluster(DevModel md, ClArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ float wred[CT / 32][3];
    __shared__ double wredd[CT / 32];
    const int K = md.ns, Nc = md.Nnu, H = a.halo;
    const unsigned rank = cl_rank();
    const int d = (int)rank, lo = d * Nc, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const ClLayout L = cl_layout(Nc, H, a.nrow, a.npt);
    float2* P = reinterpret_cast<float2*>(sm) + H;
    float2* Q = reinterpret_cast<float2*>(sm + L.oQ);
    float2* DG = reinterpret_cast<float2*>(sm + L.oDG);
    float2* X = reinterpret_cast<float2*>(sm + L.oX);
    float4* XS = reinterpret_cast<float4*>(sm) + H;
    int4* D1 = reinterpret_cast<int4*>(sm + L.oD1);
    int4* D2 = reinterpret_cast<int4*>(sm + L.oD2);
    double* xch = reinterpret_cast<double*>(sm + L.oXch);
    int* xsys = reinterpret_cast<int*>(sm + L.oXch + 8 * sizeof(double));
    const unsigned sm_base = sh_addr(sm);

    // this state's coefficient rows (FP32 pairs (-c, -c) and double-float (hi, lo) of +c) and
    // point descriptors.  D1 (FP32 pass): x = row byte offset, y = byte offset of the neighbour
    // relative to the element's own slot of P, or for a point in another state the cluster
    // address of that CTA's P slot of element 0 plus that offset; z = tab32 column of a second
    // mode or -1; w = second mode | (1 << 8 for another state).  D2: the same for XS (16-byte
    // slots).
    const int k0 = md.rbeg[d], np = md.rbeg[d + 1] - k0;
    const int row0 = np > 0 ? md.wdesc[k0].x / 8 : 0;
    {
        float2* R32 = reinterpret_cast<float2*>(sm + L.oR32);
        float2* RD = reinterpret_cast<float2*>(sm + L.oRD);
        int own = 0;  // rows of this state's points: one row of n_basis entries of the primary mode each
        for (int m = 0; m < M; ++m) own += md.rcnt[d][m] * md.nb[m];
        for (int k = tid; k < own; k += CT) {
            R32[k] = md.rct[row0 + k];
            RD[k] = md.rctd[row0 + k];
        }
        for (int k = tid; k < np; k += CT) {
            const int4 w = md.wdesc[k0 + k];
            const int dp = w.w >> 8, lin = w.y;
            const int rx = w.x - 8 * row0;
            if (dp == d) {
                D1[k] = make_int4(rx, 8 * lin, w.z, w.w & 0xff);
                D2[k] = make_int4(rx, 16 * lin, w.z, w.w & 0xff);
            } else {
                const unsigned rb = cl_map(sm_base, (unsigned)dp);  // that CTA's shared memory
                D1[k] = make_int4(rx, (int)(rb + 8u * (unsigned)(H + lin)), w.z, (w.w & 0xff) | 256);
                D2[k] = make_int4(rx, (int)(rb + 16u * (unsigned)(H + lin)), w.z, (w.w & 0xff) | 256);
            }
        }
    }
    const float2* R32 = reinterpret_cast<const float2*>(sm + L.oR32);
    const float2* RD = reinterpret_cast<const float2*>(sm + L.oRD);
    unsigned xch_remote[MAXS];
#pragma unroll
    for (int c = 0; c < MAXS; ++c) xch_remote[c] = c < K ? cl_map(sh_addr(xch), (unsigned)c) : 0u;
    // mode indices of this thread's first element and of the stride CT (one carry per digit)
    int n0[MAXM], inc[MAXM];
    decode<M>(md, tid < Nc ? tid : 0, n0);
    decode<M>(md, CT % Nc, inc);  // (an element past the plane is skipped, its digits unused)
    int slot = 0;
    // block sum of three floats, then the cluster sum in rank order (identical in every CTA)
    auto csum3 = [&](float v0, float v1, float v2) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v0 += __shfl_xor_sync(0xffffffffu, v0, o);
            v1 += __shfl_xor_sync(0xffffffffu, v1, o);
            v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        }
        if (lane == 0) {
            wred[wid][0] = v0;
            wred[wid][1] = v1;
            wred[wid][2] = v2;
        }
        __syncthreads();
        float t0 = 0.f, t1 = 0.f, t2 = 0.f;
        if (lane < CT / 32) {
            t0 = wred[lane][0];
            t1 = wred[lane][1];
            t2 = wred[lane][2];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t0 += __shfl_xor_sync(0xffffffffu, t0, o);
            t1 += __shfl_xor_sync(0xffffffffu, t1, o);
            t2 += __shfl_xor_sync(0xffffffffu, t2, o);
        }
        double* my = xch + 4 * slot;
        if (tid == 0) {
            my[0] = t0;
            my[1] = t1;
            my[2] = t2;
        }
        cl_sync();
        float3 s3 = make_float3(0.f, 0.f, 0.f);
        for (int c = 0; c < K; ++c) {
            const unsigned ra = xch_remote[c] + 32u * (unsigned)slot;
            s3.x += (float)dsm_d(ra);
            s3.y += (float)dsm_d(ra + 8);
            s3.z += (float)dsm_d(ra + 16);
        }
        slot ^= 1;
        return s3;
    };
    // block sum of a float (FP32 within a warp, FP64 across warps) and the cluster sum in FP64
    auto csum_d = [&](float v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) wredd[wid] = (double)v;
        __syncthreads();
        double t = lane < CT / 32 ? wredd[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (tid == 0) xch[4 * slot] = t;
        cl_sync();
        double s = 0.0;
        for (int c = 0; c < K; ++c) s += dsm_d(xch_remote[c] + 32u * (unsigned)slot);
        slot ^= 1;
        return s;
    };
    const float* tab = md.tab32;

    for (;;) {
        // ---- next system (rank 0 draws it, every CTA reads rank 0's copy)
        if (rank == 0 && tid == 0) {
            const int q = atomicAdd(a.counter, 1);
            *xsys = q < a.nsys ? a.nsys - 1 - q : -1;
        }
        cl_sync();
        const int s = dsm_i(cl_map(sh_addr(xsys), 0u));
        if (s < 0) break;
        const int e = a.sys_e[s];
        const long long so = (long long)s * md.N + lo;  // this CTA's part of system s
        const float2* dg32 = a.diag32 + (long long)e * md.N + lo;
        const float4* dgdf = a.diagdf + (long long)e * md.N + lo;
        const double2* b = a.b64 + so;
        float4* xs = a.xs + so;
        float2 r[EPT];  // this thread's residual entries (element tid + j CT)
        int iters = 0, refines = 0, status = -1;
        double bnorm = 0.0, rn = 0.0, prev = 0.0;
        float inres = 1.f;
        for (int k = 0;; ++k) {
            // ---- refinement residual r = b - A x (double-float); x = 0 in the first round
            if (k > 0) {
                for (int i = tid; i < Nc; i += CT) XS[i] = xs[i];
                for (int i = tid; i < H; i += CT) XS[-1 - i] = XS[Nc + i] = make_float4(0.f, 0.f, 0.f, 0.f);
                cl_sync();  // every CTA's XS complete before neighbours are read across the cluster
            }
            float nrm = 0.f;
            {
                int n[MAXM];
#pragma unroll
                for (int m = 0; m < MAXM; ++m) n[m] = n0[m];
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    const int i = tid + j * CT;
                    if (j > 0) {  // advance the digits by CT
                        int c = 0;
#pragma unroll
                        for (int m = M - 1; m >= 0; --m) {
                            const int v = n[m] + inc[m] + c;
                            c = v >= md.nb[m];
                            n[m] = c ? v - md.nb[m] : v;
                        }
                    }
                    r[j] = make_float2(0.f, 0.f);
                    if (i >= Nc) continue;
                    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
                    const double2 bb = b[i];
                    if ((__double_as_longlong(bb.x) | __double_as_longlong(bb.y)) != 0) {  // b is mostly zero
                        rh = (float)bb.x;
                        ih = (float)bb.y;
                        rl = (float)(bb.x - (double)rh);
                        il = (float)(bb.y - (double)ih);
                    }
                    if (k > 0) {
                        const float4 x = XS[i], g = dgdf[i];
                        df_fma(rh, rl, -g.x, -g.z, x.x, x.z);
                        df_fma(rh, rl, g.y, g.w, x.y, x.w);
                        df_fma(ih, il, -g.x, -g.z, x.y, x.w);
                        df_fma(ih, il, -g.y, -g.w, x.x, x.z);
                        const unsigned char* xb = reinterpret_cast<const unsigned char*>(XS + i);
                        int kk = 0;
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const int kend = kk + md.rcnt[d][m];
                            const float2* row = RD + n[m];
                            for (; kk < kend; ++kk) {
                                const int4 q = D2[kk];
                                float2 c = row[q.x >> 3];
                                if (q.z >= 0) {  // a second mode's factor t (FP64 table, split hi + lo)
                                    const double tv = md.tab64[q.z + nsel<M>(n, q.w & 0xff)];
                                    const float th = (float)tv, tl = (float)(tv - (double)th);
                                    const float ph = c.x * th;
                                    c = make_float2(ph, fmaf(c.x, th, -ph) + fmaf(c.x, tl, c.y * th));
                                }
                                const float4 v = (q.w & 256) ? dsm_f4((unsigned)q.y + 16u * (unsigned)i)
                                                             : *reinterpret_cast<const float4*>(xb + q.y);
                                df_fma(rh, rl, c.x, c.y, v.x, v.z);
                                df_fma(ih, il, c.x, c.y, v.y, v.w);
                            }
                        }
                    }
                    const float2 re = df_norm(rh, rl), im = df_norm(ih, il);
                    r[j] = make_float2(re.x, im.x);
                    nrm = fmaf(re.x, re.x, fmaf(im.x, im.x, nrm));
                }
            }
            const double rr = csum_d(nrm);  // also: every CTA is done reading the others' XS
            rn = sqrt(rr);
            if (k == 0) {
                bnorm = a.bn2 ? sqrt(a.bn2[s]) : rn;
                if (bnorm == 0.0) {
                    status = VBK_SYS_ZERO_RHS;
                    rn = 0.0;
                    break;
                }
            } else {
                refines += 1;
            }
            if (!isfinite(rn)) {
                status = VBK_SYS_NAN;
                break;
            }
            if (rn <= a.tol * bnorm) {
                status = VBK_SYS_CONVERGED;
                break;
            }
            if (a.stall_check && k > 0 && !(rn <= 0.9 * prev)) {  // the FP32 inner solve no longer helps
                status = VBK_SYS_STALLED;
                break;
            }
            if (refines >= a.max_refine || iters >= a.max_iter) {
                status = VBK_SYS_MAX_ITER;
                break;
            }
            prev = rn;
            const double scale = rn;
            const float inv = (float)(1.0 / rn);
            const float target = (float)fmax(a.inner_tol, 0.3 * a.tol * bnorm / rn);
            const float target2 = target * target;
            const int icap = a.inner_cap > 0 ? (int)min((long long)a.max_iter, (long long)iters + a.inner_cap) : a.max_iter;
            // ---- inner COCG from r / ||r||: z = B^-1 r, p = z, rho = r^T z
            for (int i = tid; i < Nc; i += CT) {
                DG[i] = dg32[i];
                X[i] = make_float2(0.f, 0.f);
            }
            for (int i = tid; i < H; i += CT) P[-1 - i] = P[Nc + i] = make_float2(0.f, 0.f);
            __syncthreads();
            float rz_x = 0.f, rz_y = 0.f;
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
                const int i = tid + j * CT;
                if (i >= Nc) continue;
                r[j] = make_float2(r[j].x * inv, r[j].y * inv);
                const float2 z = a.pmode == 0 ? cdiv_f(r[j], DG[i]) : r[j];
                P[i] = z;
                rz_x += r[j].x * z.x - r[j].y * z.y;
                rz_y += r[j].x * z.y + r[j].y * z.x;
            }
            float3 t = csum3(rz_x, rz_y, 0.f);  // also: every CTA's P complete
            float2 rho = make_float2(t.x, t.y);
            float rrf = 1.f;
            const int budget = max(0, icap - iters);
            for (int it = 0; it < budget; ++it) {
                // q = A p (neighbours in other states through the cluster), p^T q
                float pq_x = 0.f, pq_y = 0.f;
                {
                    int n[MAXM];
#pragma unroll
                    for (int m = 0; m < MAXM; ++m) n[m] = n0[m];
#pragma unroll
                    for (int j = 0; j < EPT; ++j) {
                        const int i = tid + j * CT;
                        if (j > 0) {
                            int c = 0;
#pragma unroll
                            for (int m = M - 1; m >= 0; --m) {
                                const int v = n[m] + inc[m] + c;
                                c = v >= md.nb[m];
                                n[m] = c ? v - md.nb[m] : v;
                            }
                        }
                        if (i >= Nc) continue;
                        const float2 pi = P[i];
                        float2 acc = cmul<float>(DG[i], pi);
                        const unsigned char* pb = reinterpret_cast<const unsigned char*>(P + i);
                        int kk = 0;
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const int kend = kk + md.rcnt[d][m];
                            const unsigned char* row = reinterpret_cast<const unsigned char*>(R32 + n[m]);
#pragma unroll 4
                            for (; kk < kend; ++kk) {
                                const int4 q = D1[kk];
                                float2 cc = *reinterpret_cast<const float2*>(row + q.x);  // (-c, -c)
                                if (q.z >= 0) {
                                    const float f = tab[q.z + nsel<M>(n, q.w & 0xff)];
                                    cc.x *= f;
                                    cc.y *= f;
                                }
                                const float2 v = (q.w & 256) ? dsm_f2((unsigned)q.y + 8u * (unsigned)i)
                                                             : *reinterpret_cast<const float2*>(pb + q.y);
                                acc = ffma2(cc, v, acc);  // neighbours outside the basis read the zero halo
                            }
                        }
                        Q[i] = acc;
                        pq_x += pi.x * acc.x - pi.y * acc.y;
                        pq_y += pi.x * acc.y + pi.y * acc.x;
                    }
                }
                t = csum3(pq_x, pq_y, 0.f);  // also: every CTA is done reading the others' p
                const float den = t.x * t.x + t.y * t.y;
                if (!(den > 0.f) || !isfinite(den)) {
                    status = isfinite(den) ? VBK_SYS_BREAKDOWN : VBK_SYS_NAN;
                    break;
                }
                const float2 al = make_float2((rho.x * t.x + rho.y * t.y) / den, (rho.y * t.x - rho.x * t.y) / den);
                // x += alpha p, r -= alpha q, z = B^-1 r (into Q), ||r||^2, r^T z
                float rr_l = 0.f, zx = 0.f, zy = 0.f;
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    const int i = tid + j * CT;
                    if (i >= Nc) continue;
                    const float2 pi = P[i], qi = Q[i];
                    float2 xv = X[i];
                    xv.x += al.x * pi.x - al.y * pi.y;
                    xv.y += al.x * pi.y + al.y * pi.x;
                    X[i] = xv;
                    r[j].x -= al.x * qi.x - al.y * qi.y;
                    r[j].y -= al.x * qi.y + al.y * qi.x;
                    const float2 z = a.pmode == 0 ? cdiv_f(r[j], DG[i]) : r[j];
                    Q[i] = z;
                    rr_l += r[j].x * r[j].x + r[j].y * r[j].y;
                    zx += r[j].x * z.x - r[j].y * z.y;
                    zy += r[j].x * z.y + r[j].y * z.x;
                }
                t = csum3(rr_l, zx, zy);
                iters += 1;
                rrf = t.x;
                if (!isfinite(t.x) || !isfinite(t.y) || !isfinite(t.z) || t.x <= target2 || iters >= icap) break;
                const float rden = rho.x * rho.x + rho.y * rho.y;
                if (!(t.y * t.y + t.z * t.z > 0.f) || !(rden > 0.f)) {
                    status = VBK_SYS_BREAKDOWN;
                    break;
                }
                const float2 be = make_float2((t.y * rho.x + t.z * rho.y) / rden, (t.z * rho.x - t.y * rho.y) / rden);
                rho = make_float2(t.y, t.z);
                // p = z + beta p
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    const int i = tid + j * CT;
                    if (i >= Nc) continue;
                    const float2 pi = P[i], zi = Q[i];
                    P[i] = make_float2(zi.x + be.x * pi.x - be.y * pi.y, zi.y + be.x * pi.y + be.y * pi.x);
                }
                cl_sync();  // every CTA's new p complete before the next product
            }
            inres = sqrtf(rrf);
            // ---- x += scale d in double-float (this CTA's elements; scale split into hi + lo)
            {
                const float sh = (float)scale, sl = (float)(scale - (double)sh);
                for (int i = tid; i < Nc; i += CT) {
                    const float2 dv = X[i];
                    float4 v = xs[i];
                    df_fma(v.x, v.z, sh, sl, dv.x, 0.f);
                    df_fma(v.y, v.w, sh, sl, dv.y, 0.f);
                    const float2 re = df_norm(v.x, v.z), im = df_norm(v.y, v.w);
                    xs[i] = make_float4(re.x, im.x, re.y, im.y);
                }
            }
            if (status >= 0) break;  // breakdown or non-finite value in the inner solve
            __syncthreads();  // X read before the next round's staging overwrites shared memory
        }
        // ---- psi = hi + lo in FP64, and the system's record
        __syncthreads();
        double2* psi = a.psi + so;
        for (int i = tid; i < Nc; i += CT) {
            const float4 v = xs[i];
            psi[i] = make_double2(f2d_exact(v.x) + f2d_exact(v.z), f2d_exact(v.y) + f2d_exact(v.w));
        }
        if (rank == 0 && tid == 0) {
            SysState& S = a.st[s];
            S.status = status < 0 ? VBK_SYS_MAX_ITER : status;
            S.iters = iters;
            S.refines = refines;
            S.rnorm = rn;
            S.bnorm = bnorm;
            S.inres = (double)inres;
        }
    }
    cl_sync();  // no CTA leaves while another may still read its shared memory
}

template <int M, int EPT>
int cl_setup(const DevModel& md, const ClArgs& a, size_t smem, int* max_clusters) {
    auto kern = k_solve_cluster<M, EPT>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) return vbk_cuda_fail(ce, "cluster solve shared-memory opt-in");
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)md.ns;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)md.ns);
    cfg.blockDim = dim3(CT);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    ce = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (ce != cudaSuccess) return vbk_cuda_fail(ce, "cluster solve occupancy");
    *max_clusters = n;
    (void)a;
    return VBK_OK;
}

template <int M, int EPT>
cudaError_t cl_launch(const DevModel& md, const ClArgs& a, size_t smem, int nclusters, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)md.ns;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(md.ns * nclusters));
    cfg.blockDim = dim3(CT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_solve_cluster<M, EPT>, md, a);
}

int cl_ept(int Nc) { return Nc <= 8 * CT ? 8 : 16; }

}  // namespace

// Geometry of the fused cluster solve for this model, or false when it does not apply: FP32
// rows and descriptors of the one-block kernels (rok), at most 4 states (one CTA each), at most
// 16 CT unknowns per state, and the shared-memory layout within the 227 KB of one CTA.
bool vbk_cluster_plan(const DevModel& md, ClArgs* a, size_t* smem) {
    if (!md.rok || md.nsc || md.ns < 1 || md.ns > 4 || md.Nnu > 16 * CT) return false;
    int H = 0, nrow = 0, npt = 0;
    for (int d = 0; d < md.ns; ++d) {
        H = std::max(H, std::max(-md.lmin[d], md.lmax[d]));
        npt = std::max(npt, md.rbeg[d + 1] - md.rbeg[d]);
    }
    if (npt > CL_MAXPTS) return false;
    // rows of one state: the primary-mode rows of its points (largest over the states)
    for (int d = 0; d < md.ns; ++d) {
        int rows = 0;
        for (int m = 0; m < md.M; ++m) rows += md.rcnt[d][m] * md.nb[m];
        nrow = std::max(nrow, rows);
    }
    const ClLayout L = cl_layout(md.Nnu, H, nrow, npt);
    // the double-float solution overlays P, Q and DG during the residual
    if ((size_t)(md.Nnu + 2 * H) * 16 > L.oX) return false;
    if (L.bytes > 220 * 1024) return false;
    a->halo = H;
    a->nrow = nrow;
    a->npt = npt;
    *smem = L.bytes;
    return true;
}

int vbk_cluster_prepare(const DevModel& md, const ClArgs& a, size_t smem, int* max_clusters) {
    const int ept = cl_ept(md.Nnu);
    switch (md.M * 2 + (ept == 16)) {
        case 2: return cl_setup<1, 8>(md, a, smem, max_clusters);
        case 3: return cl_setup<1, 16>(md, a, smem, max_clusters);
        case 4: return cl_setup<2, 8>(md, a, smem, max_clusters);
        case 5: return cl_setup<2, 16>(md, a, smem, max_clusters);
        case 6: return cl_setup<3, 8>(md, a, smem, max_clusters);
        case 7: return cl_setup<3, 16>(md, a, smem, max_clusters);
        case 8: return cl_setup<4, 8>(md, a, smem, max_clusters);
        default: return cl_setup<4, 16>(md, a, smem, max_clusters);
    }
}

cudaError_t vbk_cluster_launch(const DevModel& md, const ClArgs& a, size_t smem, int nclusters, cudaStream_t st) {
    const int ept = cl_ept(md.Nnu);
    switch (md.M * 2 + (ept == 16)) {
        case 2: return cl_launch<1, 8>(md, a, smem, nclusters, st);
        case 3: return cl_launch<1, 16>(md, a, smem, nclusters, st);
        case 4: return cl_launch<2, 8>(md, a, smem, nclusters, st);
        case 5: return cl_launch<2, 16>(md, a, smem, nclusters, st);
        case 6: return cl_launch<3, 8>(md, a, smem, nclusters, st);
        case 7: return cl_launch<3, 16>(md, a, smem, nclusters, st);
        case 8: return cl_launch<4, 8>(md, a, smem, nclusters, st);
        default: return cl_launch<4, 16>(md, a, smem, nclusters, st);
    }
}
