// Preconditioned COCG scalars and vector updates, FP64 residual replacement,
// source construction, channel projection and the dG/dV accumulation.
//
// COCG (the CG method for the complex-symmetric matrix of Eq. 7, with the
// unconjugated bilinear form x^T y and the symmetric preconditioner P of
// Eq. 10):
//     rho_i = r_i^T z_i,  beta_i = rho_i / rho_{i-1},  p_i = z_i + beta_i p_{i-1}
//     mu_i  = p_i^T A p_i, alpha_i = rho_i / mu_i
//     x_{i+1} = x_i + alpha_i p_i,  r_{i+1} = r_i - alpha_i A p_i,  z_{i+1} = P r_{i+1}
// The scalar kernels run one thread per RHS and sum the per-CTA partials in a
// fixed order, so every RHS of a batch gets the same arithmetic as when it is
// solved alone.
#include "iobm_internal.cuh"
#include "complex_ops.cuh"

namespace iobm {

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Sum of the per-CTA partial slots of one RHS by one warp: lane l takes slots
// l, l + 32, ..., then a fixed xor-shuffle tree; the order depends only on the
// slot count, so an RHS gets the same sums alone and in any batch.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Bi-CG pairs (primary i, shadow i + pairs): rho = r~^T z from the primary's
// partials, each member's |r|^2 from its own; the pair moves through the states
// together (it is replaced when either member's residual fell by delta, it stops
// when both are below tol).
__device__ void beta_pair(RhsState* st, const double2* rho_part, const double* rr_part, int nslots,
                          int stride, int i, int pairs, int max_iter, double tol2, double delta2,
                          int mixed, int lane) {
    const int j = i + pairs;
    if (st[i].status != ST_ACTIVE) return;
    double rx = 0.0, ry = 0.0, ri = 0.0, rj = 0.0;
    for (int k = lane; k < nslots; k += 32) {
        const double2 v = rho_part[(long long)i * stride + k];
        rx += v.x;
        ry += v.y;
        ri += rr_part[(long long)i * stride + k];
        rj += rr_part[(long long)j * stride + k];
    }
    rx = warp_sum(rx);
    ry = warp_sum(ry);
    ri = warp_sum(ri);
    rj = warp_sum(rj);
    if (lane != 0) return;
    RhsState A = st[i], B = st[j];
    const double2 rho = make_double2(rx, ry);
    A.rr = ri;
    B.rr = rj;
    int to = ST_ACTIVE;
    if (!isfinite(ri) || !isfinite(rj)) {
        to = ST_BREAKDOWN;
    } else if ((ri <= tol2 * A.bb && rj <= tol2 * B.bb) ||
               (mixed && (ri <= delta2 * A.rr_ref || rj <= delta2 * B.rr_ref))) {
        to = ST_PENDING;
    } else if (A.iters >= max_iter) {
        to = ST_NOCONV;
    } else if (!finite2(rho) || (rho.x == 0.0 && rho.y == 0.0)) {
        to = ST_BREAKDOWN;
    }
    if (to == ST_ACTIVE) {
        const double2 be = A.first ? make_double2(0.0, 0.0) : cdiv(rho, A.rho);
        A.beta = B.beta = be;
        A.rho_prev = B.rho_prev = A.rho;
        A.rho = B.rho = rho;
        A.iters += 1;
        B.iters += 1;
    }
    A.status = B.status = to;
    st[i] = A;
    st[j] = B;
}

__global__ void k_beta(RhsState* st, const double2* rho_part, const double* rr_part, int nslots,
                       int stride, int nrhs, int max_iter, double tol2, double delta2, int mixed,
                       int pairs) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (pairs > 0) {
        if (i < pairs)
            beta_pair(st, rho_part, rr_part, nslots, stride, i, pairs, max_iter, tol2, delta2, mixed,
                      lane);
        return;
    }
    if (i >= nrhs) return;   // whole warps
    if (st[i].status != ST_ACTIVE) return;
    double rx = 0.0, ry = 0.0, rr = 0.0;
    for (int j = lane; j < nslots; j += 32) {
        const double2 v = rho_part[(long long)i * stride + j];
        rx += v.x;
        ry += v.y;
        rr += rr_part[(long long)i * stride + j];
    }
    rx = warp_sum(rx);
    ry = warp_sum(ry);
    rr = warp_sum(rr);
    if (lane != 0) return;
    RhsState S = st[i];
    const double2 rho = make_double2(rx, ry);
    S.rr = rr;
    if (!isfinite(rr)) {
        S.status = ST_BREAKDOWN;
    } else if (rr <= tol2 * S.bb || (mixed && rr <= delta2 * S.rr_ref)) {
        S.status = ST_PENDING;             // FP64 residual replacement / final check
    } else if (S.iters >= max_iter) {
        S.status = ST_NOCONV;
    } else if (!finite2(rho) || (rho.x == 0.0 && rho.y == 0.0)) {
        S.status = ST_BREAKDOWN;
    } else {
        S.beta = S.first ? make_double2(0.0, 0.0) : cdiv(rho, S.rho);
        S.rho_prev = S.rho;
        S.rho = rho;
        S.iters += 1;
    }
    st[i] = S;
}

__global__ void k_alpha(RhsState* st, const double2* mu_part, int nslots, int stride, int nrhs,
                        int pairs) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= (pairs > 0 ? pairs : nrhs)) return;
    if (st[i].status != ST_ACTIVE) return;
    double mx = 0.0, my = 0.0;
    for (int j = lane; j < nslots; j += 32) {
        const double2 v = mu_part[(long long)i * stride + j];
        mx += v.x;
        my += v.y;
    }
    mx = warp_sum(mx);
    my = warp_sum(my);
    if (lane != 0) return;
    RhsState S = st[i];
    const double2 mu = make_double2(mx, my);   // pairs: mu = p~^T q, the shadow's p~
    if (!finite2(mu) || (mu.x == 0.0 && mu.y == 0.0)) {
        S.status = ST_BREAKDOWN;
    } else {
        S.alpha = cdiv(S.rho, mu);
        S.pbuf ^= 1;   // the direction written by this iteration becomes current
    }
    S.first = 0;
    st[i] = S;
    if (pairs > 0) {   // the shadow takes the same alpha and status
        RhsState B = st[i + pairs];
        B.status = S.status;
        B.alpha = S.alpha;
        if (S.status != ST_BREAKDOWN) B.pbuf ^= 1;
        B.first = 0;
        st[i + pairs] = B;
    }
}

__global__ void k_restart_scalars(RhsState* st, const double2* rho_part, const double* rr_part,
                                  int nslots, int stride, int nrhs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrhs) return;
    if (st[i].status != ST_RESTART) return;
    st[i].status = ST_ACTIVE;
    (void)rho_part; (void)rr_part; (void)nslots; (void)stride;
}

cudaError_t launch_beta(RhsState* st, const double2* rho_part, const double* rr_part, int nslots,
                        int slot_stride, int nrhs, int max_iter, double tol2, double delta2,
                        int mixed, cudaStream_t s, int pairs) {
    k_beta<<<(nrhs + 3) / 4, 128, 0, s>>>(st, rho_part, rr_part, nslots, slot_stride, nrhs,
                                          max_iter, tol2, delta2, mixed, pairs);   // a warp per RHS
    return cudaGetLastError();
}
cudaError_t launch_alpha(RhsState* st, const double2* mu_part, int nslots, int slot_stride,
                         int nrhs, cudaStream_t s, int pairs) {
    k_alpha<<<(nrhs + 3) / 4, 128, 0, s>>>(st, mu_part, nslots, slot_stride, nrhs, pairs);
    return cudaGetLastError();
}

// Bi-CG cross products a_{i+pairs}^T b_i: block x of pair i sums the points of
// chunk x (equal chunks of the RHS, fixed order) into part[i][x].
template <typename T>
__global__ void k_pair_dot(const typename Cplx<T>::type* __restrict__ a,
                           const typename Cplx<T>::type* dir0, const typename Cplx<T>::type* dir1,
                           const typename Cplx<T>::type* __restrict__ b, const RhsState* st,
                           int mask, long long npts, int pairs, double2* part, int slot_stride) {
    using C = typename Cplx<T>::type;
    __shared__ double red[3 * 8];
    const int i = blockIdx.y, j = i + pairs;
    if (!((1 << st[i].status) & mask)) return;
    const C* __restrict__ av = (dir0 ? ((st[j].pbuf & 1) ? dir0 : dir1) : a) + (long long)j * npts;
    const C* __restrict__ bv = b + (long long)i * npts;
    const long long chunk = (npts + gridDim.x - 1) / gridDim.x;
    const long long k0 = blockIdx.x * chunk, k1 = min(npts, k0 + chunk);
    double re = 0.0, im = 0.0;
    for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const C u = av[k], v = bv[k];
        re += (double)u.x * v.x - (double)u.y * v.y;
        im += (double)u.x * v.y + (double)u.y * v.x;
    }
    double z = 0.0;
    block_reduce_3(re, im, z, red);
    if (threadIdx.x == 0) part[(long long)i * slot_stride + blockIdx.x] = make_double2(re, im);
}

template <typename T>
cudaError_t launch_pair_dot(const typename Cplx<T>::type* a, typename Cplx<T>::type* const* a_dir,
                            const typename Cplx<T>::type* b, const RhsState* st, int mask,
                            long long npts, int pairs, double2* part, int nslots, int slot_stride,
                            cudaStream_t s) {
    if (pairs <= 0 || nslots <= 0) return cudaSuccess;
    k_pair_dot<T><<<dim3(nslots, pairs), 256, 0, s>>>(a, a_dir ? a_dir[0] : nullptr,
                                                        a_dir ? a_dir[1] : nullptr, b, st, mask,
                                                        npts, pairs, part, slot_stride);
    return cudaGetLastError();
}
template cudaError_t launch_pair_dot<float>(const float2*, float2* const*, const float2*,
                                            const RhsState*, int, long long, int, double2*, int,
                                            int, cudaStream_t);
template cudaError_t launch_pair_dot<double>(const double2*, double2* const*, const double2*,
                                             const RhsState*, int, long long, int, double2*, int,
                                             int, cudaStream_t);

__global__ void k_gauge(double2* __restrict__ dst, const double2* __restrict__ src,
                        const double2* phx, const double2* phy, int sign, int nx, int ny,
                        long long npts) {
    const long long nxy = (long long)nx * ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts;
         i += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(i % nxy);
        double2 ph = cmul(phx[l % nx], phy[l / nx]);
        if (sign < 0) ph.y = -ph.y;
        dst[i] = cmul(ph, src[i]);
    }
}
cudaError_t launch_restart_scalars(RhsState* st, const double2* rho_part, const double* rr_part,
                                   int nslots, int slot_stride, int nrhs, cudaStream_t s) {
    k_restart_scalars<<<(nrhs + 127) / 128, 128, 0, s>>>(st, rho_part, rr_part, nslots,
                                                         slot_stride, nrhs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_axpy_update(typename Cplx<T>::type* __restrict__ x,
                              typename Cplx<T>::type* __restrict__ r,
                              typename Cplx<T>::type* p0, typename Cplx<T>::type* p1,
                              const typename Cplx<T>::type* __restrict__ q,
                              const RhsState* st, int mask, long long npts) {
    using C = typename Cplx<T>::type;
    const int rhs = blockIdx.y;
    if (!((1 << st[rhs].status) & mask)) return;
    const C al = from_d2<C>(st[rhs].alpha);
    const C* __restrict__ p = (st[rhs].pbuf & 1) ? p1 : p0;
    const long long base = (long long)rhs * npts;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts;
         i += (long long)gridDim.x * blockDim.x) {
        const long long g = base + i;
        x[g] = cfma(al, p[g], x[g]);
        r[g] = csub(r[g], cmul(al, q[g]));
    }
}

static int vec_blocks(long long npts, int cap = 1024) {
    long long b = (npts + 255) / 256;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

// per-RHS vector kernels run once per RHS in a batch (grid.y = RHS) and are
// often masked out; a modest per-RHS block count keeps the empty launches cheap
constexpr int kPerRhsBlocks = 96;

template <typename T>
cudaError_t launch_axpy_update(typename Cplx<T>::type* x, typename Cplx<T>::type* r,
                               typename Cplx<T>::type* const* pbufs,
                               const typename Cplx<T>::type* q, const RhsState* st, int mask,
                               long long npts, int nrhs, cudaStream_t s) {
    dim3 grid(vec_blocks(npts, kPerRhsBlocks), nrhs);
    k_axpy_update<T><<<grid, 256, 0, s>>>(x, r, pbufs[0], pbufs[1], q, st, mask, npts);
    return cudaGetLastError();
}
template cudaError_t launch_axpy_update<float>(float2*, float2*, float2* const*, const float2*,
                                               const RhsState*, int, long long, int, cudaStream_t);
template cudaError_t launch_axpy_update<double>(double2*, double2*, double2* const*, const double2*,
                                                const RhsState*, int, long long, int, cudaStream_t);

// Direction and operator update of the implicit operator form.  With the
// free-propagator preconditioner M = (E - T - Sigma)^{-1} the operator of Eq. 7 is
// A = M^{-1} - V - V_NL, and z = M r gives A z = r - V z - V_NL z, hence for
// p = z + beta p_old:  q = A p = (r - V z) + beta q_old - V_NL z.  One CTA per
// (plane, RHS); mu = p^T q partial per plane.  The V_NL z term is applied by the
// same CTA at the union-of-supports points of its plane, from the projections
// kb.sp computed before the launch, once the streaming part has stored p and q.
template <typename C, typename T>
__device__ __forceinline__ void pq_point(const C zv, const C rv, const T v, const C* pold,
                                         const C* qold, bool first, C be, C& pv, C& qv) {
    qv.x = rv.x - v * zv.x;
    qv.y = rv.y - v * zv.y;
    if (first) {
        pv = zv;
    } else {
        pv = cfma(be, *pold, zv);
        qv = cfma(be, *qold, qv);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_pq_update(const typename Cplx<T>::type* __restrict__ z,
                                                   const typename Cplx<T>::type* __restrict__ r,
                                                   typename Cplx<T>::type* p0,
                                                   typename Cplx<T>::type* p1,
                                                   typename Cplx<T>::type* __restrict__ q,
                                                   const T* __restrict__ V, const RhsState* st,
                                                   int mask, int nxy, long long npts,
                                                   double2* mu_part, int slot_stride,
                                                   const KbArgs<T> kb) {
    using C = typename Cplx<T>::type;
    __shared__ double red[3 * 8];
    const int rhs = blockIdx.y;
    const RhsState& S = st[rhs];
    if (!((1 << S.status) & mask)) return;
    const bool first = S.first != 0;
    const C be = from_d2<C>(S.beta);
    const long long off = (long long)rhs * npts + (long long)blockIdx.x * nxy;
    const C* __restrict__ pold = ((S.pbuf & 1) ? p1 : p0) + off;
    C* __restrict__ pnew = ((S.pbuf & 1) ? p0 : p1) + off;
    const C* __restrict__ zp = z + off;
    const C* __restrict__ rp = r + off;
    C* __restrict__ qp = q + off;
    const T* __restrict__ Vp = V + (long long)blockIdx.x * nxy;
    T mre = 0, mim = 0;
    if (sizeof(T) == 4 && (nxy & 1) == 0) {
        // two complex FP32 values per 16-byte access (every plane starts 16-byte aligned)
        const int n2 = nxy >> 1;
        for (int j = threadIdx.x; j < n2; j += blockDim.x) {
            const float4 z4 = reinterpret_cast<const float4*>(zp)[j];
            const float4 r4 = reinterpret_cast<const float4*>(rp)[j];
            const float2 v2 = reinterpret_cast<const float2*>(Vp)[j];
            float4 po4 = make_float4(0.f, 0.f, 0.f, 0.f), qo4 = po4;
            if (!first) {
                po4 = reinterpret_cast<const float4*>(pold)[j];
                qo4 = reinterpret_cast<const float4*>(qp)[j];
            }
            C pa, qa, pb, qb;
            const C poa = {po4.x, po4.y}, pob = {po4.z, po4.w};
            const C qoa = {qo4.x, qo4.y}, qob = {qo4.z, qo4.w};
            pq_point<C, T>(C{z4.x, z4.y}, C{r4.x, r4.y}, (T)v2.x, &poa, &qoa, first, be, pa, qa);
            pq_point<C, T>(C{z4.z, z4.w}, C{r4.z, r4.w}, (T)v2.y, &pob, &qob, first, be, pb, qb);
            reinterpret_cast<float4*>(pnew)[j] = make_float4(pa.x, pa.y, pb.x, pb.y);
            reinterpret_cast<float4*>(qp)[j] = make_float4(qa.x, qa.y, qb.x, qb.y);
            mre += pa.x * qa.x - pa.y * qa.y;
            mim += pa.x * qa.y + pa.y * qa.x;
            mre += pb.x * qb.x - pb.y * qb.y;
            mim += pb.x * qb.y + pb.y * qb.x;
        }
    } else {
        for (int j = threadIdx.x; j < nxy; j += blockDim.x) {
            C pv, qv;
            pq_point<C, T>(zp[j], rp[j], Vp[j], pold + j, qp + j, first, be, pv, qv);
            pnew[j] = pv;
            qp[j] = qv;
            mre += pv.x * qv.x - pv.y * qv.y;
            mim += pv.x * qv.y + pv.y * qv.x;
        }
    }
    if (kb.nproj > 0) {
        const int u0 = kb.uplane[blockIdx.x], u1 = kb.uplane[blockIdx.x + 1];
        if (u0 < u1) {   // uniform over the CTA
            __syncthreads();   // this CTA's p and q stores are visible to all its threads
            const C* __restrict__ S = kb.sp + (long long)rhs * kb.nproj;
            const int gbase = blockIdx.x * nxy;
            for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
                const int g = kb.uidx[u] - gbase;
                C acc = czero<C>();
                for (int e = kb.uptr[u]; e < kb.uptr[u + 1]; ++e)
                    acc = caxpy(kb.uval[e], S[kb.uproj[e]], acc);
                if (kb.rhs_sign) {   // left projector p(r) exp(-i s kappa.r)
                    C ph = kb.gph[g];
                    if (kb.rhs_sign[rhs] > 0) ph.y = -ph.y;
                    acc = cmul(ph, acc);
                }
                qp[g] = csub(qp[g], acc);
                const C pv = pnew[g];
                mre -= pv.x * acc.x - pv.y * acc.y;
                mim -= pv.x * acc.y + pv.y * acc.x;
            }
        }
    }
    double a0 = mre, a1 = mim, a2 = 0.0;
    block_reduce_3(a0, a1, a2, red);
    if (threadIdx.x == 0) mu_part[(long long)rhs * slot_stride + blockIdx.x] = make_double2(a0, a1);
}

template <typename T>
cudaError_t launch_pq_update(const typename Cplx<T>::type* z, const typename Cplx<T>::type* r,
                             typename Cplx<T>::type* const* pbufs, typename Cplx<T>::type* q,
                             const T* V, const RhsState* st, int mask, int nx, int ny, int nz,
                             int nrhs, double2* mu_part, int slot_stride, const KbArgs<T>& kb,
                             cudaStream_t s) {
    const int nxy = nx * ny;
    const long long npts = (long long)nxy * nz;
    if (kb.nproj > 0 && (!kb.sp || !kb.uplane)) return cudaErrorInvalidValue;
    const int threads = nxy >= 4096 ? 256 : 128;
    dim3 grid(nz, nrhs);
    k_pq_update<T><<<grid, threads, 0, s>>>(z, r, pbufs[0], pbufs[1], q, V, st, mask, nxy, npts,
                                            mu_part, slot_stride, kb);
    return cudaGetLastError();
}
template cudaError_t launch_pq_update<float>(const float2*, const float2*, float2* const*, float2*,
                                             const float*, const RhsState*, int, int, int, int,
                                             int, double2*, int, const KbArgs<float>&, cudaStream_t);
template cudaError_t launch_pq_update<double>(const double2*, const double2*, double2* const*,
                                              double2*, const double*, const RhsState*, int, int,
                                              int, int, int, double2*, int, const KbArgs<double>&,
                                              cudaStream_t);

__global__ void k_fold(double2* __restrict__ x64, float2* __restrict__ x32, const RhsState* st,
                       int mask, long long npts) {
    const int rhs = blockIdx.y;
    if (!((1 << st[rhs].status) & mask)) return;
    const long long base = (long long)rhs * npts;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 v = x32[base + i];
        double2 w = x64[base + i];
        w.x += v.x;
        w.y += v.y;
        x64[base + i] = w;
        x32[base + i] = make_float2(0.f, 0.f);
    }
}

cudaError_t launch_fold(double2* x64, float2* x32, const RhsState* st, int mask, long long npts,
                        int nrhs, cudaStream_t s) {
    dim3 grid(vec_blocks(npts, kPerRhsBlocks), nrhs);
    k_fold<<<grid, 256, 0, s>>>(x64, x32, st, mask, npts);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// r = b - y in FP64, b(l, d) = coef[d] exp(sign i G.r_l) on the entry planes.
__device__ __forceinline__ double2 source_value(const RhsDesc& D, const double2* phx,
                                                const double2* phy, int nx, int ny, int nz, int nf,
                                                int k, int ix, int iy) {
    int d = -1;
    if (D.side == 0) {
        if (k < nf) d = k;
    } else {
        if (k >= nz - nf) d = nz - 1 - k;
    }
    if (d < 0) return make_double2(0.0, 0.0);
    const double2 ex = phx[(int)(((long long)D.kx * ix) % nx)];
    const double2 ey = phy[(int)(((long long)D.ky * iy) % ny)];
    double2 ph = cmul(ex, ey);   // exp(+i G.r)
    switch (D.profile) {
        case PROF_COS: ph = make_double2(ph.x, 0.0); break;
        case PROF_SIN: ph = make_double2(ph.y, 0.0); break;
        case PROF_EXP_MINUS: ph.y = -ph.y; break;
        default: break;
    }
    return cmul(D.coef[d], ph);
}

// r = b - y (or r = b when y is null) and per-CTA partials of ||r||^2.  The points
// of each RHS are dealt to its CTAs in chunks of 256, round robin, so every CTA
// gets the same share of interior and end-plane points.  Interior points take
// r = -y by sign flips alone (no FP64 arithmetic, which GB300 runs at a small
// fraction of its FP32 rate); the N_f end planes at either end add the source b
// (nonzero on the incident side's planes only) and, with yend, the self-energy
// terms computed apart (y + yend: the same sum the self-energy forms in place).
// The squares are summed per thread in FP32 (an estimate of the norm needs no
// more) and across the CTA in FP64.
__device__ __forceinline__ double2 dneg2(double2 v) {
    return make_double2(__hiloint2double(__double2hiint(v.x) ^ (int)0x80000000, __double2loint(v.x)),
                        __hiloint2double(__double2hiint(v.y) ^ (int)0x80000000, __double2loint(v.y)));
}

__device__ __noinline__ double2 end_residual(const double2* __restrict__ y, const double2* __restrict__ yend,
                                             const RhsDesc* __restrict__ Dp, const double2* phx,
                                             const double2* phy,
                                             int nx, int ny, int nz, int nf, int rhs, long long base,
                                             long long i) {
    const int plane = nx * ny;
    const int k = (int)(i / plane);
    const int lat = (int)(i - (long long)k * plane);
    double2 yv = make_double2(0.0, 0.0);
    if (y) {
        yv = y[base + i];
        if (yend) {
            const int end = k < nf ? 0 : 1;
            const int d = end == 0 ? k : nz - 1 - k;
            yv = cadd(yv, yend[((long long)(rhs * 2 + end) * nf + d) * plane + lat]);
        }
    }
    const RhsDesc& D = *Dp;
    const bool src = (D.side == 0) ? (k < nf) : (k >= nz - nf);
    if (src) {
        const int iy = lat / nx, ix = lat - iy * nx;
        const double2 b = source_value(D, phx, phy, nx, ny, nz, nf, k, ix, iy);
        return y ? csub(b, yv) : b;
    }
    return y ? dneg2(yv) : make_double2(0.0, 0.0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_residual(const double2* __restrict__ y, double2* __restrict__ r64,
                                                  typename Cplx<T>::type* __restrict__ rT,
                                                  const RhsDesc* desc, const double2* phx,
                                                  const double2* phy, int nx, int ny, int nz, int nf,
                                                  const RhsState* st, int mask, double* rr_part,
                                                  int stride, const double2* __restrict__ yend) {
    using C = typename Cplx<T>::type;
    __shared__ double red[3 * 8];
    const int rhs = blockIdx.y;
    if (st && !((1 << st[rhs].status) & mask)) return;
    const long long plane = (long long)nx * ny;
    const long long n = plane * nz;
    const long long base = (long long)rhs * n;
    const long long e0 = (long long)nf * plane, e1 = n - e0;   // interior points [e0, e1)
    const long long step = (long long)gridDim.x * blockDim.x;
    float acc = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
        double2 v;
        if (i >= e0 && i < e1) v = y ? dneg2(y[base + i]) : make_double2(0.0, 0.0);
        else v = end_residual(y, yend, desc + rhs, phx, phy, nx, ny, nz, nf, rhs, base, i);
        if (r64) r64[base + i] = v;
        const C c = from_d2<C>(v);
        if (rT) rT[base + i] = c;
        const float fx = (float)c.x, fy = (float)c.y;
        acc = fmaf(fx, fx, fmaf(fy, fy, acc));
    }
    double a0 = acc, z1 = 0.0, z2 = 0.0;
    block_reduce_3(a0, z1, z2, red);
    if (threadIdx.x == 0) rr_part[(long long)rhs * stride + blockIdx.x] = a0;
}

constexpr int kResidualBlocks = 128;   // CTAs per RHS (fewer when the RHS has fewer slots)

template <typename T>
cudaError_t launch_residual(const double2* y, double2* r64, typename Cplx<T>::type* rT,
                            const RhsDesc* desc, const double2* phx, const double2* phy,
                            int nx, int ny, int nz, int nf, const RhsState* st, int mask,
                            double* rr_part, int slot_stride, int nrhs, cudaStream_t s,
                            int* nslots_out, const double2* yend) {
    const int blocks = slot_stride < kResidualBlocks ? slot_stride : kResidualBlocks;
    if (blocks < 1) return cudaErrorInvalidValue;
    dim3 grid(blocks, nrhs);
    k_residual<T><<<grid, 256, 0, s>>>(y, r64, rT, desc, phx, phy, nx, ny, nz, nf, st, mask,
                                       rr_part, slot_stride, yend);
    if (nslots_out) *nslots_out = blocks;
    return cudaGetLastError();
}
template cudaError_t launch_residual<float>(const double2*, double2*, float2*, const RhsDesc*,
                                            const double2*, const double2*, int, int, int, int,
                                            const RhsState*, int, double*, int, int, cudaStream_t,
                                            int*, const double2*);
template cudaError_t launch_residual<double>(const double2*, double2*, double2*, const RhsDesc*,
                                             const double2*, const double2*, int, int, int, int,
                                             const RhsState*, int, double*, int, int, cudaStream_t,
                                             int*, const double2*);

// init = 1: record ||b||^2 and start every RHS; init = 0: assess the FP64
// residual of the PENDING RHS; init = 2: record the residual of RHS that stopped.
// pairs > 0, init = 0: the FP64 check of a Bi-CG pair, both members together
__device__ void check_pair(RhsState* st, const double* rr_part, int nslots, int stride, int i,
                           int pairs, double tol2) {
    const int j = i + pairs;
    RhsState A = st[i], B = st[j];
    if (A.status != ST_PENDING) return;
    double ri = 0.0, rj = 0.0;
    for (int k = 0; k < nslots; ++k) {
        ri += rr_part[(long long)i * stride + k];
        rj += rr_part[(long long)j * stride + k];
    }
    A.res64 = sqrt(ri / A.bb);
    B.res64 = sqrt(rj / B.bb);
    A.replacements += 1;
    B.replacements += 1;
    int to;
    if (ri <= tol2 * A.bb && rj <= tol2 * B.bb) {
        to = ST_CONVERGED;
    } else if (!isfinite(ri) || !isfinite(rj)) {
        to = ST_BREAKDOWN;
    } else {
        A.rr_ref = ri;
        B.rr_ref = rj;
        to = ST_RESTART;
    }
    A.status = B.status = to;
    st[i] = A;
    st[j] = B;
}

__global__ void k_check(RhsState* st, const double* rr_part, int nslots, int stride, int nrhs,
                        double tol2, int init, int pairs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (pairs > 0 && init == 0) {
        if (i < pairs) check_pair(st, rr_part, nslots, stride, i, pairs, tol2);
        return;
    }
    if (i >= nrhs) return;
    RhsState S = st[i];
    double rr = 0.0;
    if (init == 1) {
        for (int j = 0; j < nslots; ++j) rr += rr_part[(long long)i * stride + j];
        S.bb = rr;
        S.rr_ref = rr;
        S.rr = rr;
        S.res64 = 1.0;
        S.iters = 0;
        S.replacements = 0;
        S.first = 1;
        S.pbuf = 0;
        S.beta = make_double2(0.0, 0.0);
        S.rho = make_double2(0.0, 0.0);
        S.status = (rr > 0.0) ? ST_RESTART : ST_CONVERGED;
        if (rr == 0.0) S.res64 = 0.0;
    } else if (init == 2) {
        // record the FP64 residual of RHS that stopped without converging
        if (S.status == ST_CONVERGED || S.status == ST_IDLE) return;
        for (int j = 0; j < nslots; ++j) rr += rr_part[(long long)i * stride + j];
        S.res64 = sqrt(rr / S.bb);
        if (S.status != ST_BREAKDOWN) S.status = ST_NOCONV;
    } else {
        if (S.status != ST_PENDING) return;
        for (int j = 0; j < nslots; ++j) rr += rr_part[(long long)i * stride + j];
        S.res64 = sqrt(rr / S.bb);
        S.replacements += 1;
        if (rr <= tol2 * S.bb) {
            S.status = ST_CONVERGED;
        } else if (!isfinite(rr)) {
            S.status = ST_BREAKDOWN;
        } else {
            S.rr_ref = rr;
            S.status = ST_RESTART;
        }
    }
    st[i] = S;
}

// status `from` -> `to` for every RHS (a warm start turns its freshly
// initialised RESTART RHS into PENDING ones for an FP64 residual replacement)
__global__ void k_set_status(RhsState* st, int nrhs, int from, int to) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nrhs && st[i].status == from) st[i].status = to;
}

cudaError_t launch_set_status(RhsState* st, int nrhs, int from, int to, cudaStream_t s) {
    k_set_status<<<(nrhs + 127) / 128, 128, 0, s>>>(st, nrhs, from, to);
    return cudaGetLastError();
}

cudaError_t launch_check(RhsState* st, const double* rr_part, int nslots, int slot_stride,
                         int nrhs, double tol2, int init, cudaStream_t s, int pairs) {
    k_check<<<(nrhs + 127) / 128, 128, 0, s>>>(st, rr_part, nslots, slot_stride, nrhs, tol2, init,
                                               pairs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Channel projection (Eq. 19 on the N_f outermost planes of both ends):
// out[rhs][o][side][d] = (1/N_xy) sum_l exp(-i G_o . r_l) psi(l, plane(side, d))
// for every open channel o of the RHS's energy.  FP64 throughout.
__global__ void k_projection(const double2* __restrict__ psi, const RhsDesc* desc,
                             const int* open_ptr, const int2* open_bins, const double2* phx,
                             const double2* phy, int nx, int ny, int nz, int nf, int max_open,
                             double2* out) {
    __shared__ double red[2 * kMaxNf * 2][8];
    const int o = blockIdx.x;
    const int rhs = blockIdx.y;
    const int e = desc[rhs].energy;
    const int nopen = open_ptr[e + 1] - open_ptr[e];
    if (o >= nopen) return;
    const int2 bin = open_bins[open_ptr[e] + o];
    const long long plane = (long long)nx * ny;
    const long long npts = plane * nz;
    const double2* P = psi + (long long)rhs * npts;
    double acc[2 * kMaxNf][2];
    for (int s = 0; s < 2 * kMaxNf; ++s) acc[s][0] = acc[s][1] = 0.0;
    for (int l = threadIdx.x; l < (int)plane; l += blockDim.x) {
        const int iy = l / nx, ix = l - iy * nx;
        double2 ph = cmul(phx[(int)(((long long)bin.x * ix) % nx)], phy[(int)(((long long)bin.y * iy) % ny)]);
        ph.y = -ph.y;   // exp(-i G.r)
        for (int side = 0; side < 2; ++side) {
            for (int d = 0; d < nf; ++d) {
                const int k = side == 0 ? d : nz - 1 - d;
                const double2 v = cmul(ph, P[(long long)k * plane + l]);
                acc[side * kMaxNf + d][0] += v.x;
                acc[side * kMaxNf + d][1] += v.y;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = 0; s < 2 * kMaxNf; ++s) {
        for (int c = 0; c < 2; ++c) {
            double v = acc[s][c];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0) red[s * 2 + c][warp] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * kMaxNf * 2) {
        double v = 0.0;
        for (int w = 0; w < nw; ++w) v += red[threadIdx.x][w];
        const int s = threadIdx.x >> 1, c = threadIdx.x & 1;
        const int side = s / kMaxNf, d = s % kMaxNf;
        if (d < nf) {
            double* dst = reinterpret_cast<double*>(
                out + (((long long)rhs * max_open + o) * 2 + side) * kMaxNf + d);
            dst[c] = v / (double)plane;
        }
    }
}

cudaError_t launch_projection(const double2* psi, const RhsDesc* desc, const int* open_ptr,
                              const int2* open_bins, const double2* phx, const double2* phy,
                              int nx, int ny, int nz, int nf, int max_open, double2* out,
                              int nrhs, cudaStream_t s) {
    if (max_open <= 0) return cudaSuccess;
    dim3 grid(max_open, nrhs);
    k_projection<<<grid, 256, 0, s>>>(psi, desc, open_ptr, open_bins, phx, phy, nx, ny, nz, nf,
                                      max_open, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// dG/dV(r) = sum_{o,i} 2 (v_o / v_i) Re[conj(t_oi) lambda_o(r) psi_i(r)], with the
// forward waves psi_i = sum_k B[i][k] X_k and the adjoint waves
// lambda_o = sum_j L[o][j] Y_j combined from the solved real-profile RHS; the
// host folds C[o][i] = (v_o / v_i) conj(t_oi) into U = C B.
__global__ void k_gradient(const double2* __restrict__ X, int nX, const double2* __restrict__ Y,
                           int nY, const double2* __restrict__ U, const double2* __restrict__ L,
                           int n, long long npts, double* g) {
    extern __shared__ double2 sh[];
    double2* Us = sh;
    double2* Ls = sh + (size_t)n * nX;
    for (int i = threadIdx.x; i < n * nX; i += blockDim.x) Us[i] = U[i];
    for (int i = threadIdx.x; i < n * nY; i += blockDim.x) Ls[i] = L[i];
    __syncthreads();
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < npts;
         r += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int o = 0; o < n; ++o) {
            double2 u = make_double2(0.0, 0.0), l = make_double2(0.0, 0.0);
            for (int k = 0; k < nX; ++k) u = cfma(Us[o * nX + k], X[(long long)k * npts + r], u);
            for (int j = 0; j < nY; ++j) l = cfma(Ls[o * nY + j], Y[(long long)j * npts + r], l);
            acc += 2.0 * (l.x * u.x - l.y * u.y);
        }
        g[r] = acc;
    }
}

cudaError_t launch_gradient(const double2* X, int nX, const double2* Y, int nY, const double2* U,
                            const double2* L, int n, long long npts, double* g, cudaStream_t s) {
    const size_t smem = sizeof(double2) * (size_t)n * (nX + nY);
    if (smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(k_gradient, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
    }
    k_gradient<<<vec_blocks(npts), 256, smem, s>>>(X, nX, Y, nY, U, L, n, npts, g);
    return cudaGetLastError();
}

__global__ void k_combine(double2* __restrict__ dst, const double2* __restrict__ x1, double2 c1,
                          const double2* __restrict__ x2, double2 c2, long long npts) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts;
         i += (long long)gridDim.x * blockDim.x) {
        double2 v = cmul(c1, x1[i]);
        if (x2) v = cfma(c2, x2[i], v);
        dst[i] = v;
    }
}

cudaError_t launch_gauge(double2* dst, const double2* src, const double2* phx, const double2* phy,
                         int sign, int nx, int ny, int nz, cudaStream_t s) {
    const long long npts = (long long)nx * ny * nz;
    k_gauge<<<vec_blocks(npts), 256, 0, s>>>(dst, src, phx, phy, sign, nx, ny, npts);
    return cudaGetLastError();
}

cudaError_t launch_combine(double2* dst, const double2* x1, double2 c1, const double2* x2,
                           double2 c2, long long npts, cudaStream_t s) {
    k_combine<<<vec_blocks(npts), 256, 0, s>>>(dst, x1, c1, x2, c2, npts);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Loop condition of one junction in a batched solve (the WHILE node around its
// chunk of iterations): continue while any RHS is ACTIVE, PENDING or
// RESTART and fewer than max_chunks chunks have run.  The chunk counter makes
// the loop end even if a status never settles.
__global__ void k_batch_cond(cudaGraphConditionalHandle cond, const RhsState* st, int nrhs,
                             int* counter, int max_chunks) {
    __shared__ int live;
    if (threadIdx.x == 0) live = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nrhs; i += blockDim.x) {
        const int s = st[i].status;
        if (s == ST_ACTIVE || s == ST_PENDING || s == ST_RESTART) live = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int c = *counter + 1;
        *counter = c;
        cudaGraphSetConditional(cond, (live && c < max_chunks) ? 1u : 0u);
    }
}

// IF-node condition: 1 when some RHS has a status bit in `mask`
__global__ void k_status_cond(cudaGraphConditionalHandle cond, const RhsState* st, int nrhs,
                              int mask) {
    int any = 0;
    for (int i = threadIdx.x; i < nrhs; i += blockDim.x) any |= (1 << st[i].status) & mask;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) cudaGraphSetConditional(cond, any ? 1u : 0u);
}

cudaError_t launch_status_cond(cudaGraphConditionalHandle cond, const RhsState* st, int nrhs,
                               int mask, cudaStream_t s) {
    k_status_cond<<<1, 256, 0, s>>>(cond, st, nrhs, mask);
    return cudaGetLastError();
}

cudaError_t launch_batch_cond(cudaGraphConditionalHandle cond, const RhsState* st, int nrhs,
                              int* counter, int max_chunks, cudaStream_t s) {
    k_batch_cond<<<1, 256, 0, s>>>(cond, st, nrhs, counter, max_chunks);
    return cudaGetLastError();
}

}  // namespace iobm
