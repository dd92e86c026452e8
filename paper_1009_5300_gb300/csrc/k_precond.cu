// Lateral-Fourier free-propagator preconditioner
//     z = M r,   M = (E - T - H~)^{-1}
// where T is the FD kinetic operator (Eq. 1) and H~ the jellium self-energy on
// the end planes (Eqs. 7-2, 18-2).  The paper's preconditioner (Eq. 10) is a
// truncated real-space Green's function of the Laplacian meant to approximate
// [E - H_T - H~]^{-1}; here the approximation is the exact Green's function of
// the potential-free transition region, which the lateral Fourier transform of
// Eq. 19 diagonalises: per lateral mode nu it is a banded z-system of
// bandwidth N_f whose LU factors are the same on every plane except the last
// N_f (eliminating a plane of the left lead reproduces the lead), so one
// application costs two plane-FFT passes and one forward/backward z-sweep.
//
// Kernels: (1) forward 2D FFT of every plane of r (one CTA per plane, shared
// memory ping-pong Stockham passes over all lines at once); (2) per-mode
// z-sweeps in place on the spectrum (one thread per mode, coalesced across
// modes); (3) inverse 2D FFT of every plane, fused with the Krylov dot
// products r^T z and |r|^2 of that plane.
#include "iobm_internal.cuh"
#include "complex_ops.cuh"

namespace iobm {

// one R-point butterfly of a Stockham pass (see the line FFT in k_boundary.cu)
template <typename C, int R>
__device__ __forceinline__ void stockham_bfly(const C* src, int ss, C* dst, int ds, int N, int Ns,
                                              int j, const C* __restrict__ tw, bool inv) {
    const int NR = N / R;
    const int k = j % Ns;
    const int tscale = N / (Ns * R);
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        C u = src[(j + r * NR) * ss];
        if (r) {
            C w = tw[(r * k * tscale) % N];
            if (inv) w.y = -w.y;
            u = cmul(u, w);
        }
        v[r] = u;
    }
    C o[R];
    if constexpr (R == 2) {
        o[0] = cadd(v[0], v[1]);
        o[1] = csub(v[0], v[1]);
    } else if constexpr (R == 4) {
        C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        C a2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        C a3;
        if (inv) { a3.x = -d.y; a3.y = d.x; } else { a3.x = d.y; a3.y = -d.x; }
        o[0] = cadd(a0, a2);
        o[2] = csub(a0, a2);
        o[1] = cadd(a1, a3);
        o[3] = csub(a1, a3);
    } else {
#pragma unroll
        for (int aa = 0; aa < R; ++aa) {
            C acc = v[0];
#pragma unroll
            for (int b = 1; b < R; ++b) {
                C w = tw[((aa * b) % R) * NR];
                if (inv) w.y = -w.y;
                acc = cfma(v[b], w, acc);
            }
            o[aa] = acc;
        }
    }
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * Ns) * ds] = o[r];
}

template <typename C>
__device__ __forceinline__ void bfly_dispatch(int R, const C* src, int ss, C* dst, int ds, int N,
                                              int Ns, int j, const C* tw, bool inv) {
    switch (R) {
        case 2: stockham_bfly<C, 2>(src, ss, dst, ds, N, Ns, j, tw, inv); break;
        case 3: stockham_bfly<C, 3>(src, ss, dst, ds, N, Ns, j, tw, inv); break;
        case 4: stockham_bfly<C, 4>(src, ss, dst, ds, N, Ns, j, tw, inv); break;
        case 5: stockham_bfly<C, 5>(src, ss, dst, ds, N, Ns, j, tw, inv); break;
        default: break;
    }
}

// 2D FFT of an ny x nx plane held in a (x fastest); b is a same-size scratch.
// Every pass spreads the butterflies of all lines over the whole CTA.
// Returns the buffer that holds the result.
template <typename C>
__device__ C* fft2_block(C* a, C* b, const FftAxis& ax, const FftAxis& ay, const C* twx,
                         const C* twy, bool inv) {
    const int nx = ax.n, ny = ay.n;
    C* cur = a;
    C* oth = b;
    int Ns = 1;
    for (int p = 0; p < ax.npass; ++p) {
        const int R = ax.radix[p];
        const int per = nx / R;
        for (int t = threadIdx.x; t < ny * per; t += blockDim.x) {
            const int row = t / per, j = t - row * per;
            bfly_dispatch(R, cur + row * nx, 1, oth + row * nx, 1, nx, Ns, j, twx, inv);
        }
        __syncthreads();
        C* s = cur; cur = oth; oth = s;
        Ns *= R;
    }
    Ns = 1;
    for (int p = 0; p < ay.npass; ++p) {
        const int R = ay.radix[p];
        const int per = ny / R;
        for (int t = threadIdx.x; t < nx * per; t += blockDim.x) {
            const int col = t / per, j = t - col * per;
            bfly_dispatch(R, cur + col, nx, oth + col, nx, ny, Ns, j, twy, inv);
        }
        __syncthreads();
        C* s = cur; cur = oth; oth = s;
        Ns *= R;
    }
    return cur;
}

template <typename T>
__global__ void __launch_bounds__(256) k_plane_fft_fwd(const PrecondArgs<T> a) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int plane = blockIdx.x, rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    const int nxy = a.nx * a.ny;
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + nxy;
    const long long off = (long long)rhs * a.npts + (long long)plane * nxy;
    for (int i = threadIdx.x; i < nxy; i += blockDim.x) A[i] = a.r[off + i];
    __syncthreads();
    C* res = fft2_block(A, B, a.ax, a.ay, a.twx, a.twy, false);
    for (int i = threadIdx.x; i < nxy; i += blockDim.x) a.spec[off + i] = res[i];
}

// z-sweeps of one lateral mode: forward substitution with the constant band
// multipliers over planes 0 .. nz-nf-1, a dense nf x nf solve on the last nf
// planes, backward substitution with the constant band rows.  In place.
template <typename T, int NF>
__global__ void __launch_bounds__(64) k_zsolve(const PrecondArgs<T> a) {
    using C = typename Cplx<T>::type;
    const int rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    const int nxy = a.nx * a.ny;
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= nxy) return;
    const int e = a.rhs_energy ? a.rhs_energy[rhs] : 0;
    const C* __restrict__ pc = a.pc + ((size_t)e * nxy + mode) * kPcStrideDev;
    C l[NF + 1], u[NF + 1], S2[NF * NF];
#pragma unroll
    for (int j = 1; j <= NF; ++j) l[j] = pc[j - 1];
#pragma unroll
    for (int j = 0; j <= NF; ++j) u[j] = pc[NF + j];
#pragma unroll
    for (int i = 0; i < NF * NF; ++i) S2[i] = pc[2 * NF + 1 + i];
    const C uinv = cdivc(make_one<C>(), u[0]);
    const int nz = a.nz, m = nz - NF;
    C* __restrict__ s = a.spec + (long long)rhs * a.npts + mode;
    const T scale = (T)1 / (T)nxy;   // the forward FFT above carries no 1/N_xy
    // forward: y_k = r_k - sum_j l_j y_{k-j}
    C hist[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) hist[j] = czero<C>();   // hist[j] = y_{k-1-j}
    for (int k = 0; k < m; ++k) {
        C y = cscale(s[(long long)k * nxy], scale);
#pragma unroll
        for (int j = 1; j <= NF; ++j) y = csub(y, cmul(l[j], hist[j - 1]));
        s[(long long)k * nxy] = y;
#pragma unroll
        for (int j = NF - 1; j > 0; --j) hist[j] = hist[j - 1];
        hist[0] = y;
    }
    // last nf planes: g_i = r_i - sum_{j: i-j < m} l_j y_{i-j};  x_2 = S2^{-1} g
    C g[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        C v = cscale(s[(long long)(m + i) * nxy], scale);
#pragma unroll
        for (int j = 1; j <= NF; ++j) {
            // y_{m+i-j} is hist[j-1-i] when m+i-j <= m-1, i.e. j > i
            if (j > i) v = csub(v, cmul(l[j], hist[j - 1 - i]));
        }
        g[i] = v;
    }
    C xl[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        C v = czero<C>();
#pragma unroll
        for (int j = 0; j < NF; ++j) v = cfma(S2[i * NF + j], g[j], v);
        xl[i] = v;
        s[(long long)(m + i) * nxy] = v;
    }
    // backward: x_k = (y_k - sum_j u_j x_{k+j}) / u_0
    C nxt[NF];   // nxt[j] = x_{k+1+j}
#pragma unroll
    for (int j = 0; j < NF; ++j) nxt[j] = xl[j];
    for (int k = m - 1; k >= 0; --k) {
        C v = s[(long long)k * nxy];
#pragma unroll
        for (int j = 1; j <= NF; ++j) v = csub(v, cmul(u[j], nxt[j - 1]));
        v = cmul(v, uinv);
        s[(long long)k * nxy] = v;
#pragma unroll
        for (int j = NF - 1; j > 0; --j) nxt[j] = nxt[j - 1];
        nxt[0] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_plane_ifft_dots(const PrecondArgs<T> a) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3 * 8];
    const int plane = blockIdx.x, rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    const int nxy = a.nx * a.ny;
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + nxy;
    const long long off = (long long)rhs * a.npts + (long long)plane * nxy;
    for (int i = threadIdx.x; i < nxy; i += blockDim.x) A[i] = a.spec[off + i];
    __syncthreads();
    C* res = fft2_block(A, B, a.ax, a.ay, a.twx, a.twy, true);
    T dre = 0, dim = 0, nrm = 0;
    for (int i = threadIdx.x; i < nxy; i += blockDim.x) {
        const C z = res[i];
        a.z[off + i] = z;
        if (a.dot_part) {
            const C r = a.r[off + i];
            dre += r.x * z.x - r.y * z.y;
            dim += r.x * z.y + r.y * z.x;
            nrm += r.x * r.x + r.y * r.y;
        }
    }
    if (a.dot_part) {
        double d0 = dre, d1 = dim, d2 = nrm;
        block_reduce_3(d0, d1, d2, red);
        if (threadIdx.x == 0) {
            a.dot_part[(long long)rhs * a.slot_stride + plane] = make_double2(d0, d1);
            a.nrm_part[(long long)rhs * a.slot_stride + plane] = d2;
        }
    }
}

template <typename T>
size_t precond_smem_bytes(int nx, int ny) {
    using C = typename Cplx<T>::type;
    return 2 * sizeof(C) * (size_t)nx * ny;
}

cudaError_t precond_prepare() {
    const int lim = 160 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_plane_fft_fwd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_plane_fft_fwd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_plane_ifft_dots<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_plane_ifft_dots<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    return e;
}

template <typename T>
cudaError_t launch_precond_fourier(const PrecondArgs<T>& a, int nrhs, cudaStream_t s) {
    const size_t smem = precond_smem_bytes<T>(a.nx, a.ny);
    if (smem > 160 * 1024) return cudaErrorInvalidValue;
    dim3 gp(a.nz, nrhs);
    k_plane_fft_fwd<T><<<gp, 256, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nxy = a.nx * a.ny;
    dim3 gz((nxy + 63) / 64, nrhs);
    switch (a.nf) {
        case 1: k_zsolve<T, 1><<<gz, 64, 0, s>>>(a); break;
        case 2: k_zsolve<T, 2><<<gz, 64, 0, s>>>(a); break;
        case 3: k_zsolve<T, 3><<<gz, 64, 0, s>>>(a); break;
        case 4: k_zsolve<T, 4><<<gz, 64, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_plane_ifft_dots<T><<<gp, 256, smem, s>>>(a);
    return cudaGetLastError();
}

template size_t precond_smem_bytes<float>(int, int);
template size_t precond_smem_bytes<double>(int, int);
template cudaError_t launch_precond_fourier<float>(const PrecondArgs<float>&, int, cudaStream_t);
template cudaError_t launch_precond_fourier<double>(const PrecondArgs<double>&, int, cudaStream_t);

}  // namespace iobm
