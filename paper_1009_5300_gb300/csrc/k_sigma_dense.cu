// The end-plane self-energy of Eq. 7 applied as a dense matrix: solver (b) of
// Sec. III, which multiplies Sigma^r(z_0) Psi(z_0) and Sigma^r(z_{N_z+1}) Psi(z_{N_z+1})
// directly at O(N_in (N_f N_xy)^2) per application, where the library's default
// (Eq. 19) diagonalises the same operator with lateral FFTs.  It exists as the
// ablation of the transform: the operator is the same up to rounding, so solves with
// either form take the same iterations and give the same transmission.
//
// The dense block between end planes d and d' is circulant in the lateral offset:
//     Sigma~[(d, r), (d', r')] = K_dd'(r - r'),
//     K_dd'(dr) = (1/N_xy) sum_nu Sigma~_nu[d][d'] exp(i G_nu . dr)
// (the inverse lateral transform of the per-mode blocks of Eq. 18-2).  The kernel K
// is formed once per energy, the N_f N_xy square matrix filled from it and kept in
// memory for the solve, as solver (b) does; the right end uses the same matrix with
// the plane order mirrored (plane nz - 1 - d).
//
// Apply: a tiled complex matrix product per electrode end, 64 matrix rows x 16 RHS
// per CTA, k-steps of 32 staged in shared memory; RHS of one tile that belong to
// different energies are taken in separate passes over their energy's matrix.
#include "iobm_internal.cuh"
#include "complex_ops.cuh"

#include <algorithm>

namespace iobm {

// K[e][d][d'][dy][dx], FP64, from the per-mode blocks sigma[e][ky][kx][d][d']
__global__ void k_sigma_kernel(const double2* __restrict__ sigma, const double2* __restrict__ twx,
                               const double2* __restrict__ twy, int nx, int ny, int nf, int ne,
                               double2* __restrict__ K) {
    const int nxy = nx * ny;
    const long long n = (long long)ne * nf * nf * nxy;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int off = (int)(idx % nxy);
        const long long ed = idx / nxy;          // (e nf + d) nf + d'
        const int dd = (int)(ed % (nf * nf));
        const int e = (int)(ed / (nf * nf));
        const int dx = off % nx, dy = off / nx;
        const double2* S = sigma + (size_t)e * nxy * nf * nf + dd;
        double2 acc = make_double2(0.0, 0.0);
        for (int ky = 0; ky < ny; ++ky) {
            const double2 wy = cconj(twy[(ky * dy) % ny]);   // exp(+2 pi i ky dy / ny)
            for (int kx = 0; kx < nx; ++kx) {
                const double2 w = cmul(wy, cconj(twx[(kx * dx) % nx]));
                acc = cfma(S[((size_t)ky * nx + kx) * nf * nf], w, acc);
            }
        }
        K[idx] = cscale(acc, 1.0 / nxy);
    }
}

// D[e][(d, r)][(d', r')] = K[e][d][d'][r - r'] in the working precision
template <typename C>
__global__ void k_sigma_dense_fill(const double2* __restrict__ K, int nx, int ny, int nf, int ne,
                                   C* __restrict__ D) {
    const int nxy = nx * ny;
    const long long M = (long long)nf * nxy;
    const long long n = (long long)ne * M * M;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long col = idx % M;
        const long long rem = idx / M;
        const long long row = rem % M;
        const int e = (int)(rem / M);
        const int d = (int)(row / nxy), i = (int)(row % nxy);
        const int dp = (int)(col / nxy), j = (int)(col % nxy);
        int dx = i % nx - j % nx, dy = i / nx - j / nx;
        if (dx < 0) dx += nx;
        if (dy < 0) dy += ny;
        const double2 v = K[(((size_t)e * nf + d) * nf + dp) * nxy + dy * nx + dx];
        C c;
        c.x = v.x;
        c.y = v.y;
        D[idx] = c;
    }
}

constexpr int kDenseTM = 64;    // matrix rows per CTA
constexpr int kDenseTN = 16;    // RHS per CTA
constexpr int kDenseTK = 32;    // k-step
constexpr int kDenseThreads = 256;

// y_end -= D x_end for the RHS in the mask (end = blockIdx.y, row tile blockIdx.x,
// RHS tile blockIdx.z); part[(rhs 2 + end) ntm + tile] = x_end^T (-D x_end) over the
// tile's rows when dots are wanted
template <typename T>
__global__ void __launch_bounds__(kDenseThreads) k_sigma_dense(const SigmaArgs<T> a, const typename Cplx<T>::type* __restrict__ D,
                                                               int nrhs, double2* __restrict__ part) {
    using C = typename Cplx<T>::type;
    __shared__ C As[kDenseTK][kDenseTM + 1];
    __shared__ C Bs[kDenseTK][kDenseTN];
    __shared__ const C* xs[kDenseTN];
    __shared__ int es[kDenseTN], sel[kDenseTN], todo[kDenseTN];
    __shared__ int ecur;
    __shared__ T red_re[kDenseThreads], red_im[kDenseThreads];
    const int tid = threadIdx.x;
    const int tx = tid % kDenseTN, ty = tid / kDenseTN;
    const int nxy = a.nx * a.ny;
    const int M = a.nf * nxy;
    const int ntm = (M + kDenseTM - 1) / kDenseTM;
    const int tile = blockIdx.x, end = blockIdx.y;
    const int r0 = blockIdx.z * kDenseTN;
    const int i0 = tile * kDenseTM;
    if (tid < kDenseTN) {
        const int rhs = r0 + tid;
        int act = 0;
        const C* xp = nullptr;
        int e = 0;
        if (rhs < nrhs) {
            const int st = a.state ? a.state[rhs].status : ST_ACTIVE;
            act = ((1 << st) & a.mask) != 0;
            xp = (a.pnew[0] ? a.pnew[1 - (a.state[rhs].pbuf & 1)] : a.x) + (long long)rhs * a.npts;
            e = a.rhs_energy ? a.rhs_energy[rhs] : 0;
        }
        xs[tid] = xp;
        es[tid] = e;
        todo[tid] = act;
    }
    __syncthreads();
    // row k of an end block: plane d = k / nxy (mirrored at the right end), point k mod nxy
    auto end_off = [&](int k) -> long long {
        const int d = k / nxy;
        const int plane = end ? a.nz - 1 - d : d;
        return (long long)plane * nxy + (k - d * nxy);
    };
    for (;;) {
        if (tid == 0) {
            int e = -1;
            for (int n = 0; n < kDenseTN; ++n)
                if (todo[n]) { e = es[n]; break; }
            ecur = e;
        }
        __syncthreads();
        const int e = ecur;
        if (e < 0) break;
        if (tid < kDenseTN) sel[tid] = todo[tid] && es[tid] == e;
        __syncthreads();
        const C* __restrict__ De = D + (size_t)e * M * M;
        C acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = czero<C>();
        for (int k0 = 0; k0 < M; k0 += kDenseTK) {
#pragma unroll
            for (int j = 0; j < (kDenseTM * kDenseTK) / kDenseThreads; ++j) {
                const int idx = tid + j * kDenseThreads;
                const int r = idx / kDenseTK, c = idx % kDenseTK;
                const int row = i0 + r, k = k0 + c;
                As[c][r] = (row < M && k < M) ? De[(size_t)row * M + k] : czero<C>();
            }
#pragma unroll
            for (int j = 0; j < (kDenseTN * kDenseTK) / kDenseThreads; ++j) {
                const int idx = tid + j * kDenseThreads;
                const int kk = idx % kDenseTK, n = idx / kDenseTK;
                const int k = k0 + kk;
                Bs[kk][n] = (sel[n] && k < M) ? xs[n][end_off(k)] : czero<C>();
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < kDenseTK; ++kk) {
                const C b = Bs[kk][tx];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = cfma(As[kk][ty * 4 + q], b, acc[q]);
            }
            __syncthreads();
        }
        // y_end -= D x_end, and the x^T (-D x) partial of the tile's rows
        T pre = 0, pim = 0;
        if (sel[tx]) {
            const int rhs = r0 + tx;
            C* __restrict__ y = a.y + (long long)rhs * a.npts;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = i0 + ty * 4 + q;
                if (row < M) {
                    const long long o = end_off(row);
                    y[o] = csub(y[o], acc[q]);
                    const C xv = xs[tx][o];
                    pre -= xv.x * acc[q].x - xv.y * acc[q].y;
                    pim -= xv.x * acc[q].y + xv.y * acc[q].x;
                }
            }
        }
        if (part) {
            red_re[tid] = pre;
            red_im[tid] = pim;
            __syncthreads();
            if (tid < kDenseTN && sel[tid]) {
                double sre = 0.0, sim = 0.0;
                for (int t = 0; t < kDenseThreads / kDenseTN; ++t) {   // fixed order
                    sre += (double)red_re[t * kDenseTN + tid];
                    sim += (double)red_im[t * kDenseTN + tid];
                }
                part[((long long)(r0 + tid) * 2 + end) * ntm + tile] = make_double2(sre, sim);
            }
        }
        if (tid < kDenseTN && sel[tid]) todo[tid] = 0;
        __syncthreads();
    }
}

// the self-energy's mu slots of each RHS in the mask: the sum of each end's tile
// partials in the end's first slot, zeros in the others (nslots per end)
__global__ void k_sigma_dense_slots(const SigmaArgs<double> meta, const RhsState* st, int mask,
                                    const double2* __restrict__ part, int ntm, int nrhs, int nslots_end) {
    const int rhs = blockIdx.x;
    if (rhs >= nrhs) return;
    if (st && !((1 << st[rhs].status) & mask)) return;
    for (int s = threadIdx.x; s < 2 * nslots_end; s += blockDim.x) {
        const int end = s / nslots_end;
        double2 v = make_double2(0.0, 0.0);
        if (s % nslots_end == 0)
            for (int t = 0; t < ntm; ++t) {   // fixed order
                const double2 p = part[((long long)rhs * 2 + end) * ntm + t];
                v.x += p.x;
                v.y += p.y;
            }
        meta.dot_part[(long long)rhs * meta.slot_stride + meta.slot_base + s] = v;
    }
}

int dense_row_tiles(int nf, int nxy) { return (nf * nxy + kDenseTM - 1) / kDenseTM; }

cudaError_t build_sigma_dense(const double2* sigma, const double2* twx, const double2* twy, int nx,
                              int ny, int nf, int ne, double2* kscratch, float2* d32, double2* d64,
                              cudaStream_t s) {
    const long long nk = (long long)ne * nf * nf * nx * ny;
    const int bk = (int)std::min<long long>((nk + 255) / 256, 65535);
    k_sigma_kernel<<<bk, 256, 0, s>>>(sigma, twx, twy, nx, ny, nf, ne, kscratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (d64) k_sigma_dense_fill<double2><<<4096, 256, 0, s>>>(kscratch, nx, ny, nf, ne, d64);
    if (d32) k_sigma_dense_fill<float2><<<4096, 256, 0, s>>>(kscratch, nx, ny, nf, ne, d32);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sigma_dense(const SigmaArgs<T>& a, const typename Cplx<T>::type* D, int nrhs,
                               double2* part, int nslots_end, cudaStream_t s) {
    if (nrhs <= 0) return cudaSuccess;
    const int ntm = dense_row_tiles(a.nf, a.nx * a.ny);
    dim3 grid(ntm, 2, (nrhs + kDenseTN - 1) / kDenseTN);
    double2* p = a.dot_part ? part : nullptr;
    k_sigma_dense<T><<<grid, kDenseThreads, 0, s>>>(a, D, nrhs, p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !a.dot_part) return e;
    SigmaArgs<double> meta{};
    meta.dot_part = a.dot_part;
    meta.slot_stride = a.slot_stride;
    meta.slot_base = a.slot_base;
    k_sigma_dense_slots<<<nrhs, 64, 0, s>>>(meta, a.state, a.mask, part, ntm, nrhs, nslots_end);
    return cudaGetLastError();
}

template cudaError_t launch_sigma_dense<float>(const SigmaArgs<float>&, const float2*, int, double2*, int,
                                               cudaStream_t);
template cudaError_t launch_sigma_dense<double>(const SigmaArgs<double>&, const double2*, int, double2*,
                                                int, cudaStream_t);

}  // namespace iobm
