// Boundary self-energy through lateral 2D FFTs (Eqs. 8, 18-1, 18-2, 19) and the
// Kleinman-Bylander nonlocal term.
//
// Self-energy: one thread-block cluster of N_f CTAs per (RHS, electrode end).
// CTA d loads the operand plane at depth d into shared memory and transforms
// it with a mixed-radix Stockham FFT (one warp per line, rows then columns;
// the forward transform carries the 1/N_xy of Eq. 19).  After a cluster
// barrier every CTA reads the N_f spectra of its cluster through distributed
// shared memory and forms, per lateral mode nu, sum_d' Sigma~_nu[d][d'] psi~_nu(d')
// (for N_f = 1 this is the diagonal product of Eq. 18-2), transforms back and
// subtracts the result from the operator output on its plane (or, for the FP64
// residual, stores -Sigma x in an end-plane buffer of its own, so that it can run
// beside the stencil that writes the operator output).  The unconjugated product
// x^T (-Sigma x) over the plane goes to a dot slot.
//
// KB term: one CTA per RHS.  Warps first form s_p = dvol * sum_r p(r) x(r) for
// every projector (fixed per-lane order plus a fixed shuffle tree), then the
// CTA walks the union of the supports point by point and subtracts
// sum_p E_p p(r) s_p, so the result does not depend on scheduling.
#include <cooperative_groups.h>

#include "iobm_internal.cuh"
#include "complex_ops.cuh"
#include "fft_ct.cuh"
#include "fft_line.cuh"

namespace cg = cooperative_groups;

namespace iobm {

// 2D FFT of an ny x nx plane (x fastest) in shared memory.  scratch: per warp
// max(nx, ny) elements.
template <typename C>
__device__ void fft2(C* plane, C* scratch, const FftAxis& ax, const FftAxis& ay,
                     const C* __restrict__ twx, const C* __restrict__ twy, bool inv) {
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nx = ax.n, ny = ay.n;
    const int smax = nx > ny ? nx : ny;
    const int pitch = nx + 1;   // padded rows: column lines do not share one bank
    C* my = scratch + warp * smax;
    for (int row = warp; row < ny; row += nwarps) fft_line(plane + row * pitch, 1, my, ax, twx, inv, lane);
    __syncthreads();
    for (int col = warp; col < nx; col += nwarps) fft_line(plane + col, pitch, my, ay, twy, inv, lane);
    __syncthreads();
}

constexpr int kSigmaPer = 16;   // lateral modes per thread in the multiply step
constexpr int kSigmaMaxThreads = 256;
constexpr size_t kSigmaMaxSmem = 200 * 1024;

template <typename T>
size_t sigma_smem_bytes(int nx, int ny, int threads) {
    using C = typename Cplx<T>::type;
    const int smax = nx > ny ? nx : ny;
    return sizeof(C) * ((size_t)(nx + 1) * ny + (size_t)(threads / 32) * smax) + 3 * 32 * sizeof(double);
}

template <typename T>
__global__ void __launch_bounds__(kSigmaMaxThreads) k_sigma(const SigmaArgs<T> a) {
    using C = typename Cplx<T>::type;
    cg::cluster_group cluster = cg::this_cluster();
    const int d = blockIdx.x;         // depth of this CTA's plane (= rank in cluster)
    const int end = blockIdx.y;       // 0 left, 1 right
    const int rhs = blockIdx.z;
    const int st = a.state ? a.state[rhs].status : ST_ACTIVE;
    if (!((1 << st) & a.mask)) return;   // uniform over the cluster

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = a.nx, ny = a.ny, nf = a.nf;
    const int nxy = nx * ny;
    const int smax = nx > ny ? nx : ny;
    const int pitch = nx + 1;
    C* buf = reinterpret_cast<C*>(smem_raw);   // [ny][pitch]
    C* scratch = buf + ny * pitch;
    double* red = reinterpret_cast<double*>(scratch + (blockDim.x / 32) * smax);

    const int plane = (end == 0) ? d : (a.nz - 1 - d);
    const long long off = (long long)rhs * a.npts + (long long)plane * nxy;
    const C* xb = a.pnew[0] ? a.pnew[1 - (a.state[rhs].pbuf & 1)] : a.x;
    const C* __restrict__ X = xb + off;
    for (int i = threadIdx.x; i < nxy; i += blockDim.x) buf[(i / nx) * pitch + (i % nx)] = X[i];
    __syncthreads();
    fft2(buf, scratch, a.ax, a.ay, a.twx, a.twy, false);

    cluster.sync();   // every spectrum of the cluster is complete

    const int e = a.rhs_energy ? a.rhs_energy[rhs] : 0;
    const C* __restrict__ S = a.sigma + (size_t)e * nxy * nf * nf;
    const T inv_n = (T)1 / (T)nxy;
    C out[kSigmaPer];
#pragma unroll
    for (int j = 0; j < kSigmaPer; ++j) {
        const int m = threadIdx.x + j * blockDim.x;
        C acc = czero<C>();
        if (m < nxy) {
            const int sm = (m / nx) * pitch + (m % nx);
            for (int dp = 0; dp < nf; ++dp) {
                const C* remote = cluster.map_shared_rank(buf, dp);
                acc = cfma(S[((size_t)m * nf + d) * nf + dp], remote[sm], acc);
            }
            acc = cscale(acc, inv_n);
        }
        out[j] = acc;
    }
    cluster.sync();   // all remote reads done before spectra are overwritten
#pragma unroll
    for (int j = 0; j < kSigmaPer; ++j) {
        const int m = threadIdx.x + j * blockDim.x;
        if (m < nxy) buf[(m / nx) * pitch + (m % nx)] = out[j];
    }
    __syncthreads();
    fft2(buf, scratch, a.ax, a.ay, a.twx, a.twy, true);

    C* __restrict__ Y = a.y + off;
    C* __restrict__ YE = a.yend ? a.yend + ((long long)(rhs * 2 + end) * nf + d) * nxy : nullptr;
    T tre = 0, tim = 0;   // per-thread partials in the working precision
    for (int i = threadIdx.x; i < nxy; i += blockDim.x) {
        const C s = buf[(i / nx) * pitch + (i % nx)];
        const C xv = X[i];
        if (YE) YE[i] = cneg(s);
        else Y[i] = csub(Y[i], s);
        tre -= xv.x * s.x - xv.y * s.y;
        tim -= xv.x * s.y + xv.y * s.x;
    }
    double sre = tre, sim = tim, dummy = 0.0;
    if (a.dot_part) {
        block_reduce_3(sre, sim, dummy, red);
        if (threadIdx.x == 0)
            a.dot_part[(long long)rhs * a.slot_stride + a.slot_base + end * nf + d] =
                make_double2(sre, sim);
    }
}

// The same cluster scheme for square N x N planes with a compile-time FFT plan:
// 256 threads spread every butterfly pass over all lines of the plane, each
// thread keeps its operand points in registers for the closing dot product.
constexpr int kSigmaCtThreads = 256;

template <typename T, int N>
__global__ void __launch_bounds__(kSigmaCtThreads) k_sigma_ct(const SigmaArgs<T> a) {
    using C = typename Cplx<T>::type;
    cg::cluster_group cluster = cg::this_cluster();
    const int d = blockIdx.x;
    const int end = blockIdx.y;
    const int rhs = blockIdx.z;
    const int st = a.state ? a.state[rhs].status : ST_ACTIVE;
    if (!((1 << st) & a.mask)) return;   // uniform over the cluster

    constexpr int NXY = N * N;
    constexpr int PT = CtPitch<N>::P;
    constexpr int PER = (NXY + kSigmaCtThreads - 1) / kSigmaCtThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* A = reinterpret_cast<C*>(smem_raw);   // [N][PT] spectrum (the result of ct_fft2 lands here)
    C* B = A + N * PT;                       // ping-pong scratch
    C* tw = B + N * PT;
    __shared__ double red[3 * (kSigmaCtThreads / 32)];
    const int nf = a.nf;
    for (int i = threadIdx.x; i < N; i += kSigmaCtThreads) tw[i] = a.twx[i];

    const int plane = (end == 0) ? d : (a.nz - 1 - d);
    const long long off = (long long)rhs * a.npts + (long long)plane * NXY;
    const C* xb = a.pnew[0] ? a.pnew[1 - (a.state[rhs].pbuf & 1)] : a.x;
    const C* __restrict__ X = xb + off;
    C* __restrict__ Y = a.y + off;
    C xv[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int i = threadIdx.x + j * kSigmaCtThreads;
        if (i < NXY) {
            xv[j] = X[i];
            A[(i / N) * PT + (i % N)] = xv[j];
        }
    }
    __syncthreads();
    ct_fft2<C, N, kSigmaCtThreads>(A, B, tw, false);   // an even number of passes: the spectrum is in A

    cluster.sync();   // every spectrum of the cluster is complete

    const int e = a.rhs_energy ? a.rhs_energy[rhs] : 0;
    const C* __restrict__ S = a.sigma + (size_t)e * NXY * nf * nf;
    const T inv_n = (T)1 / (T)NXY;
    C out[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int m = threadIdx.x + j * kSigmaCtThreads;
        C acc = czero<C>();
        if (m < NXY) {
            const int sm = (m / N) * PT + (m % N);
            const C* Sm = S + ((size_t)m * nf + d) * nf;
            for (int dp = 0; dp < nf; ++dp) {
                const C* remote = cluster.map_shared_rank(A, dp);
                acc = cfma(Sm[dp], remote[sm], acc);
            }
            acc = cscale(acc, inv_n);
        }
        out[j] = acc;
    }
    cluster.sync();   // all remote reads done before the spectra are overwritten
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int m = threadIdx.x + j * kSigmaCtThreads;
        if (m < NXY) A[(m / N) * PT + (m % N)] = out[j];
    }
    __syncthreads();
    ct_fft2<C, N, kSigmaCtThreads>(A, B, tw, true);

    C* __restrict__ YE = a.yend ? a.yend + ((long long)(rhs * 2 + end) * nf + d) * NXY : nullptr;
    T tre = 0, tim = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int i = threadIdx.x + j * kSigmaCtThreads;
        if (i < NXY) {
            const C sv = A[(i / N) * PT + (i % N)];
            if (YE) YE[i] = cneg(sv);
            else Y[i] = csub(Y[i], sv);
            tre -= xv[j].x * sv.x - xv[j].y * sv.y;
            tim -= xv[j].x * sv.y + xv[j].y * sv.x;
        }
    }
    if (a.dot_part) {
        double sre = tre, sim = tim, dummy = 0.0;
        block_reduce_3(sre, sim, dummy, red);
        if (threadIdx.x == 0)
            a.dot_part[(long long)rhs * a.slot_stride + a.slot_base + end * nf + d] =
                make_double2(sre, sim);
    }
}

template <typename T, int N>
size_t sigma_ct_smem_bytes() {
    using C = typename Cplx<T>::type;
    return sizeof(C) * (2 * (size_t)N * CtPitch<N>::P + N);
}

static bool sigma_ct_size(int nx, int ny) {
    return nx == ny && (nx == 12 || nx == 16 || nx == 24 || nx == 32 || nx == 48 || nx == 64);
}

static int sigma_threads(int nxy) {
    int t = (nxy + kSigmaPer - 1) / kSigmaPer;
    t = ((t + 31) / 32) * 32;
    if (t < 128) t = 128;
    return t;   // <= kSigmaMaxThreads when nxy <= 4096 (checked on the host)
}

template <typename T>
cudaError_t launch_sigma(const SigmaArgs<T>& a, int nrhs, cudaStream_t s) {
    const int nxy = a.nx * a.ny;
    if (nxy > kSmemPlaneLimit) {
        if (!a.scratch) return cudaErrorInvalidValue;
        return launch_sigma_large<T>(a, nrhs, s);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nf, 2, nrhs);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.nf;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (sigma_ct_size(a.nx, a.ny)) {
        cfg.blockDim = dim3(kSigmaCtThreads, 1, 1);
        switch (a.nx) {
#define IOBM_SIG(NN)                                              \
            case NN:                                              \
                cfg.dynamicSmemBytes = sigma_ct_smem_bytes<T, NN>(); \
                return cudaLaunchKernelEx(&cfg, k_sigma_ct<T, NN>, a);
            IOBM_SIG(12) IOBM_SIG(16) IOBM_SIG(24) IOBM_SIG(32) IOBM_SIG(48) IOBM_SIG(64)
#undef IOBM_SIG
            default: return cudaErrorInvalidValue;
        }
    }
    const int threads = sigma_threads(nxy);
    if (threads > kSigmaMaxThreads) return cudaErrorInvalidValue;
    const size_t smem = sigma_smem_bytes<T>(a.nx, a.ny, threads);
    if (smem > kSigmaMaxSmem) return cudaErrorInvalidValue;
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    return cudaLaunchKernelEx(&cfg, k_sigma<T>, a);
}

// ---------------------------------------------------------------------------
// KB nonlocal term, y -= sum_p |p> E_p dvol <p|x>, in two kernels: the
// projections (one CTA per (projector, group of kKbRhs RHS), the support split
// over the CTA's threads and reduced in a fixed order) into a [rhs][projector]
// scratch, then the application over the union of supports (one thread per
// union point and RHS group) with the partials of the dot product x'^T (-V_NL x)
// per CTA.  The index tables are loaded once per RHS group and the operand
// gathers of the group's RHS are in flight together.
constexpr int kKbProjThreads = 128;
constexpr int kKbBatch = 4;            // support points per thread and RHS in flight
constexpr int kKbApplyThreads = 256;
constexpr int kKbRhs = 4;              // RHS per CTA

int kb_slots(int nunion) { return (nunion + kKbApplyThreads - 1) / kKbApplyThreads; }

// exp(i s kappa.r_l) from gph[l] = exp(i kappa.r_l), s = +1 or -1
template <typename C>
__device__ __forceinline__ C bloch_phase(const C* gph, int l, int s) {
    C g = gph[l];
    if (s < 0) g.y = -g.y;
    return g;
}

template <typename T>
__device__ __forceinline__ bool kb_rhs_live(const KbArgs<T>& a, int rhs, int nrhs) {
    if (rhs >= nrhs) return false;
    const int st = a.state ? a.state[rhs].status : ST_ACTIVE;
    return ((1 << st) & a.mask) != 0;
}

template <typename T>
__global__ void __launch_bounds__(kKbProjThreads) k_kb_proj(const KbArgs<T> a, int nrhs) {
    using C = typename Cplx<T>::type;
    __shared__ double red[2 * kKbRhs][kKbProjThreads / 32];
    const int p = blockIdx.x, r0 = blockIdx.y * kKbRhs;
    bool live[kKbRhs];
    const C* X[kKbRhs];
    bool any = false;
#pragma unroll
    for (int j = 0; j < kKbRhs; ++j) {
        live[j] = kb_rhs_live(a, r0 + j, nrhs);
        any |= live[j];
        X[j] = nullptr;
        if (live[j]) {
            const int rhs = r0 + j;
            const C* xb = a.zsrc ? a.zsrc
                                 : (a.pnew[0] ? a.pnew[1 - (a.state[rhs].pbuf & 1)] : a.x);
            X[j] = xb + (long long)rhs * a.npts;   // projected operand
        }
    }
    if (!any) return;
    const int e0 = a.pptr[p], e1 = a.pptr[p + 1];
    T tre[kKbRhs], tim[kKbRhs];
#pragma unroll
    for (int j = 0; j < kKbRhs; ++j) tre[j] = tim[j] = 0;
    for (int i0 = e0 + threadIdx.x; i0 < e1; i0 += kKbProjThreads * kKbBatch) {
        int idx[kKbBatch];
        T v[kKbBatch];
#pragma unroll
        for (int u = 0; u < kKbBatch; ++u) {
            const int i = i0 + kKbProjThreads * u;
            idx[u] = (i < e1) ? a.pidx[i] : -1;
            v[u] = (i < e1) ? a.pval[i] : (T)0;
        }
        C xv[kKbRhs][kKbBatch];
#pragma unroll
        for (int j = 0; j < kKbRhs; ++j)
#pragma unroll
            for (int u = 0; u < kKbBatch; ++u)
                xv[j][u] = (live[j] && idx[u] >= 0) ? X[j][idx[u]] : czero<C>();
        if (a.rhs_sign) {   // right projector p(r) exp(i s kappa.r) (gauge of a Bloch vector)
#pragma unroll
            for (int j = 0; j < kKbRhs; ++j) {
                const int sj = live[j] ? a.rhs_sign[r0 + j] : 1;
#pragma unroll
                for (int u = 0; u < kKbBatch; ++u)
                    if (live[j] && idx[u] >= 0)
                        xv[j][u] = cmul(bloch_phase(a.gph, idx[u] % a.nxy, sj), xv[j][u]);
            }
        }
#pragma unroll
        for (int j = 0; j < kKbRhs; ++j)
#pragma unroll
            for (int u = 0; u < kKbBatch; ++u) {
                tre[j] += v[u] * xv[j][u].x;
                tim[j] += v[u] * xv[j][u].y;
            }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kKbRhs; ++j) {
        double re = tre[j], im = tim[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_down_sync(0xffffffffu, re, o);
            im += __shfl_down_sync(0xffffffffu, im, o);
        }
        if (lane == 0) {
            red[2 * j][warp] = re;
            red[2 * j + 1][warp] = im;
        }
    }
    __syncthreads();
    if (threadIdx.x < kKbRhs && live[threadIdx.x]) {
        const int j = threadIdx.x;
        double sr = 0.0, si = 0.0;
        for (int w = 0; w < kKbProjThreads / 32; ++w) {
            sr += red[2 * j][w];
            si += red[2 * j + 1][w];
        }
        const double f = a.coupling[p] * a.dvol;
        a.sp[(long long)(r0 + j) * a.nproj + p] = from_d2<C>(make_double2(sr * f, si * f));
    }
}

template <typename T>
__global__ void __launch_bounds__(kKbApplyThreads) k_kb_apply(const KbArgs<T> a, int nrhs) {
    using C = typename Cplx<T>::type;
    __shared__ double red[3 * (kKbApplyThreads / 32)];
    const int r0 = blockIdx.y * kKbRhs;
    bool live[kKbRhs];
    bool any = false;
#pragma unroll
    for (int j = 0; j < kKbRhs; ++j) {
        live[j] = kb_rhs_live(a, r0 + j, nrhs);
        any |= live[j];
    }
    if (!any) return;
    const int u = blockIdx.x * kKbApplyThreads + threadIdx.x;
    const bool in = u < a.nunion;
    const int g = in ? a.uidx[u] : 0;
    const int eb = in ? a.uptr[u] : 0, ee = in ? a.uptr[u + 1] : 0;
    C yv[kKbRhs], dv[kKbRhs], acc[kKbRhs];
#pragma unroll
    for (int j = 0; j < kKbRhs; ++j) {
        yv[j] = dv[j] = acc[j] = czero<C>();
        if (in && live[j]) {
            const int rhs = r0 + j;
            const long long base = (long long)rhs * a.npts;
            yv[j] = a.y[base + g];
            if (a.dot_part) {
                const C* xb = a.pnew[0] ? a.pnew[1 - (a.state[rhs].pbuf & 1)] : a.x;
                dv[j] = xb[base + g];   // dot operand
            }
        }
    }
    for (int e = eb; e < ee; ++e) {
        const T v = a.uval[e];
        const int pj = a.uproj[e];
#pragma unroll
        for (int j = 0; j < kKbRhs; ++j)
            if (live[j]) acc[j] = caxpy(v, a.sp[(long long)(r0 + j) * a.nproj + pj], acc[j]);
    }
    if (a.rhs_sign && in) {   // left projector p(r) exp(-i s kappa.r)
#pragma unroll
        for (int j = 0; j < kKbRhs; ++j)
            if (live[j]) acc[j] = cmul(bloch_phase(a.gph, g % a.nxy, -a.rhs_sign[r0 + j]), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < kKbRhs; ++j) {
        if (in && live[j]) a.y[(long long)(r0 + j) * a.npts + g] = csub(yv[j], acc[j]);
        if (a.dot_part && live[j]) {   // uniform over the CTA
            double dre = -(double)(dv[j].x * acc[j].x - dv[j].y * acc[j].y);
            double dim = -(double)(dv[j].x * acc[j].y + dv[j].y * acc[j].x);
            double dummy = 0.0;
            block_reduce_3(dre, dim, dummy, red);
            if (threadIdx.x == 0)
                a.dot_part[(long long)(r0 + j) * a.slot_stride + a.slot_base + blockIdx.x] =
                    make_double2(dre, dim);
            __syncthreads();   // red is reused by the next RHS
        }
    }
}

template <typename T>
cudaError_t launch_kb_proj(const KbArgs<T>& a, int nrhs, cudaStream_t s) {
    if (a.nproj == 0) return cudaSuccess;
    if (!a.sp) return cudaErrorInvalidValue;
    const int groups = (nrhs + kKbRhs - 1) / kKbRhs;
    k_kb_proj<T><<<dim3(a.nproj, groups), kKbProjThreads, 0, s>>>(a, nrhs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kb(const KbArgs<T>& a, int nrhs, cudaStream_t s) {
    if (a.nproj == 0) return cudaSuccess;
    if (!a.sp) return cudaErrorInvalidValue;
    const int groups = (nrhs + kKbRhs - 1) / kKbRhs;
    k_kb_proj<T><<<dim3(a.nproj, groups), kKbProjThreads, 0, s>>>(a, nrhs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.nunion == 0) return cudaSuccess;
    k_kb_apply<T><<<dim3(kb_slots(a.nunion), groups), kKbApplyThreads, 0, s>>>(a, nrhs);
    return cudaGetLastError();
}

// One-time attribute set-up (outside any stream capture): the self-energy
// kernel may use up to kSigmaMaxSmem bytes of dynamic shared memory.
cudaError_t sigma_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_sigma<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSigmaMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sigma<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSigmaMaxSmem);
#define IOBM_SIG(NN)                                                                              \
    if (e == cudaSuccess)                                                                         \
        e = cudaFuncSetAttribute(k_sigma_ct<float, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)sigma_ct_smem_bytes<float, NN>());                          \
    if (e == cudaSuccess)                                                                         \
        e = cudaFuncSetAttribute(k_sigma_ct<double, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)sigma_ct_smem_bytes<double, NN>());
    IOBM_SIG(12) IOBM_SIG(16) IOBM_SIG(24) IOBM_SIG(32) IOBM_SIG(48) IOBM_SIG(64)
#undef IOBM_SIG
    return e;
}

template size_t sigma_smem_bytes<float>(int, int, int);
template size_t sigma_smem_bytes<double>(int, int, int);
template cudaError_t launch_sigma<float>(const SigmaArgs<float>&, int, cudaStream_t);
template cudaError_t launch_sigma<double>(const SigmaArgs<double>&, int, cudaStream_t);
template cudaError_t launch_kb_proj<float>(const KbArgs<float>&, int, cudaStream_t);
template cudaError_t launch_kb_proj<double>(const KbArgs<double>&, int, cudaStream_t);
template cudaError_t launch_kb<float>(const KbArgs<float>&, int, cudaStream_t);
template cudaError_t launch_kb<double>(const KbArgs<double>&, int, cudaStream_t);

}  // namespace iobm
