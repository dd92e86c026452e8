// Lateral plane FFTs (Eq. 19) for planes larger than one CTA's shared memory
// holds (more than 4096 points, up to 256 x 256): the 2D transform as two
// passes over global memory, first along x (CTAs of kLargeRows whole rows),
// then along y (CTAs of kLargeCols whole columns), each line transformed by
// one warp with the mixed-radix Stockham line FFT.  The forward transform is
// unnormalised; the 1/N_xy of Eq. 19 is applied where the spectrum is used.
//
// Two users:
//  * the free-propagator preconditioner: row pass r -> spectrum, column pass,
//    per-mode z-sweeps (k_zsolve), inverse column pass, inverse row pass
//    spectrum -> z fused with the partials of r^T z and |r|^2;
//  * the self-energy: row and column passes over the 2 N_f end planes of the
//    operand into a compact scratch, per-mode Sigma~ mixing, inverse column
//    pass, inverse row pass fused with y -= Sigma x and the partials of
//    x^T (-Sigma x).
// Partial sums go to one slot per (plane, row block), so every sum has a
// fixed order.
#include <cooperative_groups.h>

#include "iobm_internal.cuh"
#include "complex_ops.cuh"
#include "fft_bfly.cuh"
#include "fft_line.cuh"

namespace cg = cooperative_groups;

namespace iobm {

constexpr int kLargeRows = 8;    // rows per CTA in the x pass (one warp each)
constexpr int kLargeCols = 16;   // columns per CTA in the y pass
constexpr int kLargeThreads = 256;

int large_row_blocks(int ny) { return (ny + kLargeRows - 1) / kLargeRows; }

bool large_plane_supported(int nx, int ny) { return nx <= 256 && ny <= 256; }

template <typename T>
struct LargeFftArgs {
    using C = typename Cplx<T>::type;
    const C* src;            // row pass source
    const C* srcp[2];        // if srcp[0]: source = srcp[1 - pbuf] of the RHS (COCG direction)
    C* dst;                  // row pass destination (epilogue 0, 1)
    long long src_rhs, dst_rhs;   // element strides between RHS
    int src_end, dst_end;    // 1: plane index pi of the launch is end plane pi of the volume
    int nx, ny, nz, nf;
    FftAxis ax, ay;
    const C* twx;
    const C* twy;
    int inv;
    const RhsState* state;
    int mask;
    // epilogue 1: z = dst, dots with r; epilogue 2: y[end plane] -= v, dots with the operand
    const C* r;
    C* y;
    const C* xop;
    const C* xopp[2];
    double2* dot_part;
    double* nrm_part;
    int slot_stride, slot_base;
    long long npts;
};

// end plane pi (0 .. 2 nf - 1) of the volume: left planes by depth, then right
__device__ __forceinline__ int end_plane(int pi, int nf, int nz) {
    return pi < nf ? pi : nz - 1 - (pi - nf);
}

template <typename T, int EPI>
__global__ void __launch_bounds__(kLargeThreads) k_fft_rows_large(const LargeFftArgs<T> a) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3 * (kLargeThreads / 32)];
    const int rb = blockIdx.x, pi = blockIdx.y, rhs = blockIdx.z;
    int pbuf = 0;
    if (a.state) {
        if (!((1 << a.state[rhs].status) & a.mask)) return;
        pbuf = a.state[rhs].pbuf & 1;
    }
    const int nx = a.nx, ny = a.ny;
    const int nxy = nx * ny;
    const int r0 = rb * kLargeRows;
    const int nr = min(kLargeRows, ny - r0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C* buf = reinterpret_cast<C*>(smem_raw);          // [kLargeRows][nx]
    C* scratch = buf + kLargeRows * nx;              // [warps][nx]
    const int sp = a.src_end ? end_plane(pi, a.nf, a.nz) : pi;
    const C* sbase = a.srcp[0] ? a.srcp[1 - pbuf] : a.src;
    const C* __restrict__ S = sbase + (long long)rhs * a.src_rhs + (long long)sp * nxy + (long long)r0 * nx;
    for (int i = threadIdx.x; i < nr * nx; i += kLargeThreads) buf[i] = S[i];
    __syncthreads();
    if (warp < nr) fft_line(buf + warp * nx, 1, scratch + warp * nx, a.ax, a.twx, a.inv != 0, lane);
    __syncthreads();
    T d0 = 0, d1 = 0, d2 = 0;
    if constexpr (EPI == 0 || EPI == 1) {
        const int dp = a.dst_end ? end_plane(pi, a.nf, a.nz) : pi;
        const long long off = (long long)rhs * a.dst_rhs + (long long)dp * nxy + (long long)r0 * nx;
        C* __restrict__ D = a.dst + off;
        for (int i = threadIdx.x; i < nr * nx; i += kLargeThreads) {
            const C v = buf[i];
            D[i] = v;
            if constexpr (EPI == 1) {
                if (a.dot_part) {
                    const C rv = a.r[off + i];
                    d0 += rv.x * v.x - rv.y * v.y;
                    d1 += rv.x * v.y + rv.y * v.x;
                    d2 += rv.x * rv.x + rv.y * rv.y;
                }
            }
        }
    } else {
        // y -= Sigma x on end plane ep; partials of x^T (-Sigma x)
        const int ep = end_plane(pi, a.nf, a.nz);
        const long long off = (long long)rhs * a.npts + (long long)ep * nxy + (long long)r0 * nx;
        const C* xb = a.xopp[0] ? a.xopp[1 - pbuf] : a.xop;
        C* __restrict__ Y = a.y + off;
        const C* __restrict__ X = xb + off;
        for (int i = threadIdx.x; i < nr * nx; i += kLargeThreads) {
            const C v = buf[i];
            Y[i] = csub(Y[i], v);
            const C xv = X[i];
            d0 -= xv.x * v.x - xv.y * v.y;
            d1 -= xv.x * v.y + xv.y * v.x;
        }
    }
    if ((EPI == 1 || EPI == 2) && a.dot_part) {
        double s0 = d0, s1 = d1, s2 = d2;
        block_reduce_3(s0, s1, s2, red);
        if (threadIdx.x == 0) {
            const long long slot = (long long)rhs * a.slot_stride + a.slot_base +
                                   (long long)pi * gridDim.x + rb;
            a.dot_part[slot] = make_double2(s0, s1);
            if (EPI == 1 && a.nrm_part) a.nrm_part[slot] = s2;
        }
    }
}

// column pass in place on planes data + rhs * rhs_stride + pi * nxy
template <typename T>
__global__ void __launch_bounds__(kLargeThreads) k_fft_cols_large(typename Cplx<T>::type* data,
                                                                  long long rhs_stride, int nx, int ny,
                                                                  FftAxis ay,
                                                                  const typename Cplx<T>::type* twy,
                                                                  int inv, const RhsState* state,
                                                                  int mask) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cb = blockIdx.x, pi = blockIdx.y, rhs = blockIdx.z;
    if (state && !((1 << state[rhs].status) & mask)) return;
    constexpr int TP = kLargeCols + 1;   // padded row of the tile
    const int c0 = cb * kLargeCols;
    const int nc = min(kLargeCols, nx - c0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C* tile = reinterpret_cast<C*>(smem_raw);   // [ny][TP]
    C* scratch = tile + ny * TP;                 // [warps][ny]
    C* __restrict__ P = data + (long long)rhs * rhs_stride + (long long)pi * nx * ny + c0;
    for (int i = threadIdx.x; i < ny * nc; i += kLargeThreads) {
        const int row = i / nc, c = i - row * nc;
        tile[row * TP + c] = P[(long long)row * nx + c];
    }
    __syncthreads();
    for (int c = warp; c < nc; c += kLargeThreads / 32)
        fft_line(tile + c, TP, scratch + warp * ny, ay, twy, inv != 0, lane);
    __syncthreads();
    for (int i = threadIdx.x; i < ny * nc; i += kLargeThreads) {
        const int row = i / nc, c = i - row * nc;
        P[(long long)row * nx + c] = tile[row * TP + c];
    }
}

// out[end][d][m] = (1 / N_xy) sum_dp Sigma~_m[d][dp] in[end][dp][m], compact end-plane spectra
template <typename T>
__global__ void k_sigma_mix_large(const typename Cplx<T>::type* in, typename Cplx<T>::type* out,
                                  const typename Cplx<T>::type* sigma, const int* rhs_energy,
                                  int nxy, int nf, const RhsState* state, int mask) {
    using C = typename Cplx<T>::type;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int end = blockIdx.y, rhs = blockIdx.z;
    if (state && !((1 << state[rhs].status) & mask)) return;
    if (m >= nxy) return;
    const int e = rhs_energy ? rhs_energy[rhs] : 0;
    const C* __restrict__ Sm = sigma + ((size_t)e * nxy + m) * nf * nf;
    const long long base = (long long)rhs * 2 * nf * nxy + (long long)end * nf * nxy + m;
    const T inv_n = (T)1 / (T)nxy;
    for (int d = 0; d < nf; ++d) {
        C acc = czero<C>();
        for (int dp = 0; dp < nf; ++dp) acc = cfma(Sm[d * nf + dp], in[base + (long long)dp * nxy], acc);
        out[base + (long long)d * nxy] = cscale(acc, inv_n);
    }
}

// ---------------------------------------------------------------------------
// 128 x 128 planes (FP32) transformed on chip by a cluster of two CTAs: CTA
// rank q holds rows 64 q .. 64 q + 63 (a 66 KB tile, pitch 129).  128 = 16 x 8:
// pass 1 (rows, 16-point DFTs in registers straight from global memory), pass 2
// (rows, radix 8 after the twiddles exp(-+2 pi i r j / 128), in place per
// butterfly), then the columns: pass 3 (16-point DFTs of rows j + 8 m, half of them
// in the peer CTA's tile, read through distributed shared memory; every input is
// read before the cluster barrier, the outputs rows 16 j + a are local), pass 4
// (radix 8 on rows j + 16 r of both tiles, outputs straight to global memory).  The
// forward transform reads r and writes the spectrum; the inverse reads the spectrum
// and writes z with the r^T z and |r|^2 partials (slots plane * 16 + rank).
constexpr int kP128 = 128;
constexpr int kP128Rows = 64;                  // rows per CTA
constexpr int kP128Pitch = kP128 + 1;
constexpr int kP128Threads = 512;
constexpr size_t kP128Smem = sizeof(float2) * ((size_t)kP128Rows * kP128Pitch + kP128);

// With UPD the forward transform first applies the COCG update x += alpha p,
// r -= alpha q at the points its first pass reads (r_rw, x, the RHS's direction
// buffer p0/p1, q), and transforms the updated r.
struct Fft128Update {
    float2* x;
    float2* r;
    const float2* p[2];
    const float2* q;
};

template <bool INV, bool UPD>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kP128Threads, 2)
    k_fft128_cluster(const PrecondArgs<float> a, int slot_per_plane, const Fft128Update u) {
    using C = float2;
    constexpr int N = kP128, R1 = 16, R2 = 8, PT = kP128Pitch;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int plane = blockIdx.x >> 1, rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;   // uniform over the cluster
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3 * (kP128Threads / 32)];
    C* A = reinterpret_cast<C*>(smem_raw);             // [64][129]
    C* tw = A + kP128Rows * PT;                        // [128]
    const int tid = threadIdx.x;
    for (int i = tid; i < N; i += kP128Threads) tw[i] = a.twx[i];
    const long long off = (long long)rhs * a.npts + (long long)plane * (N * N);
    const C* __restrict__ src = (INV ? a.spec : a.r) + off;
    auto twiddled = [&](C v, int e) {
        C w = tw[e];
        if (INV) w.y = -w.y;
        return cmul(v, w);
    };
    {   // pass 1: row (64 rank + yl), 16-point DFT of columns j + 8 m
        const int j = tid % R2, yl = tid / R2;
        C v[R1], o[R1];
        const long long roff = (long long)(rank * kP128Rows + yl) * N + j;
        if constexpr (UPD) {
            const C al = from_d2<C>(a.state[rhs].alpha);
            C* __restrict__ R = u.r + off + roff;
            C* __restrict__ X = u.x + off + roff;
            const C* __restrict__ P = ((a.state[rhs].pbuf & 1) ? u.p[1] : u.p[0]) + off + roff;
            const C* __restrict__ Q = u.q + off + roff;
#pragma unroll
            for (int m = 0; m < R1; ++m) {
                const int c = m * R2;
                v[m] = csub(R[c], cmul(al, Q[c]));
                R[c] = v[m];
                X[c] = cfma(al, P[c], X[c]);
            }
        } else {
#pragma unroll
            for (int m = 0; m < R1; ++m) v[m] = src[roff + m * R2];
        }
        dft_reg<C, R1, INV>(v, o);
#pragma unroll
        for (int q = 0; q < R1; ++q) A[yl * PT + j * R1 + q] = o[q];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 2; ++k) {   // pass 2: rows, radix 8, in place per butterfly
        const int t = tid + k * kP128Threads;
        const int yl = t % kP128Rows, j = t / kP128Rows;
        C v[R2], o[R2];
        v[0] = A[yl * PT + j];
#pragma unroll
        for (int r = 1; r < R2; ++r) v[r] = twiddled(A[yl * PT + j + r * R1], r * j);
        dft_reg<C, R2, INV>(v, o);
#pragma unroll
        for (int q = 0; q < R2; ++q) A[yl * PT + j + q * R1] = o[q];
    }
    cluster.sync();   // the row transforms of both tiles are complete
    C* peer = cluster.map_shared_rank(A, rank ^ 1);
    const C* t0 = rank == 0 ? A : peer;   // rows 0-63
    const C* t1 = rank == 0 ? peer : A;   // rows 64-127
    auto at = [&](int row, int col) -> C {
        return (row < kP128Rows ? t0 : t1)[(row & (kP128Rows - 1)) * PT + col];
    };
    C o3[R1];
    const int x3 = tid % N, j3 = rank * 4 + tid / N;   // outputs rows 16 j3 .. 16 j3 + 15: local
    {   // pass 3: columns, 16-point DFT of rows j3 + 8 m (m < 8 in tile 0, m >= 8 in tile 1)
        C v[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) {
            v[m] = at(j3 + m * R2, x3);
        }
        dft_reg<C, R1, INV>(v, o3);
    }
    cluster.sync();   // every pass-3 read of both tiles is done
#pragma unroll
    for (int q = 0; q < R1; ++q) A[(j3 * R1 + q - rank * kP128Rows) * PT + x3] = o3[q];
    cluster.sync();   // pass-3 outputs of both tiles visible
    C* __restrict__ dst = (INV ? a.z : a.spec) + off;
    const C* __restrict__ rin = a.r + off;
    const bool dots = INV && a.dot_part != nullptr;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {   // pass 4: columns, radix 8 on rows j + 16 r, to global memory
        const int t = tid + k * kP128Threads;
        const int x = t % N, j = rank * 8 + t / N;
        C v[R2], o[R2];
#pragma unroll
        for (int r = 0; r < R2; ++r) {
            const C u = at(j + r * R1, x);
            v[r] = r ? twiddled(u, r * j) : u;
        }
        dft_reg<C, R2, INV>(v, o);
#pragma unroll
        for (int q = 0; q < R2; ++q) {
            const int i = (j + q * R1) * N + x;
            dst[i] = o[q];
            if (dots) {
                const C rv = rin[i];
                d0 += rv.x * o[q].x - rv.y * o[q].y;
                d1 += rv.x * o[q].y + rv.y * o[q].x;
                d2 += rv.x * rv.x + rv.y * rv.y;
            }
        }
    }
    if (dots) {
        double s0 = d0, s1 = d1, s2 = d2;
        block_reduce_3(s0, s1, s2, red);
        // the CTA's sum (held by thread 0) in slot `rank` of the plane; rank 0's threads
        // 2 .. slot_per_plane - 1 write zeros to the plane's other slots
        const long long plane_slot0 = (long long)rhs * a.slot_stride + (long long)plane * slot_per_plane;
        if (tid == 0) {
            a.dot_part[plane_slot0 + rank] = make_double2(s0, s1);
            if (a.nrm_part) a.nrm_part[plane_slot0 + rank] = s2;
        } else if (rank == 0 && tid >= 2 && tid < slot_per_plane) {
            a.dot_part[plane_slot0 + tid] = make_double2(0.0, 0.0);
            if (a.nrm_part) a.nrm_part[plane_slot0 + tid] = 0.0;
        }
    }
    cluster.sync();   // the peer's tile is not released while this CTA may still read it
}

template <typename T>
static size_t rows_smem(int nx) {
    return sizeof(typename Cplx<T>::type) * (size_t)(kLargeRows + kLargeThreads / 32) * nx;
}
template <typename T>
static size_t cols_smem(int ny) {
    return sizeof(typename Cplx<T>::type) * (size_t)ny * (kLargeCols + 1 + kLargeThreads / 32);
}

static void set128(const void* f, cudaError_t& e) {
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kP128Smem);
}

cudaError_t fft_large_prepare() {
    const int lim = 200 * 1024;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    };
    set((const void*)k_fft_rows_large<float, 0>);
    set((const void*)k_fft_rows_large<float, 1>);
    set((const void*)k_fft_rows_large<float, 2>);
    set((const void*)k_fft_rows_large<double, 0>);
    set((const void*)k_fft_rows_large<double, 1>);
    set((const void*)k_fft_rows_large<double, 2>);
    set((const void*)k_fft_cols_large<float>);
    set((const void*)k_fft_cols_large<double>);
    set128((const void*)k_fft128_cluster<false, false>, e);
    set128((const void*)k_fft128_cluster<false, true>, e);
    set128((const void*)k_fft128_cluster<true, false>, e);
    return e;
}

template <typename T, int EPI>
static cudaError_t launch_rows(const LargeFftArgs<T>& a, int nplanes, int nrhs, cudaStream_t s) {
    dim3 grid(large_row_blocks(a.ny), nplanes, nrhs);
    k_fft_rows_large<T, EPI><<<grid, kLargeThreads, rows_smem<T>(a.nx), s>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_cols(typename Cplx<T>::type* data, long long rhs_stride, int nplanes,
                               int nrhs, int nx, int ny, const FftAxis& ay,
                               const typename Cplx<T>::type* twy, int inv, const RhsState* st,
                               int mask, cudaStream_t s) {
    dim3 grid((nx + kLargeCols - 1) / kLargeCols, nplanes, nrhs);
    k_fft_cols_large<T><<<grid, kLargeThreads, cols_smem<T>(ny), s>>>(data, rhs_stride, nx, ny, ay,
                                                                      twy, inv, st, mask);
    return cudaGetLastError();
}

// preconditioner through the two-pass transforms; partial slots: nz * row blocks
template <typename T>
cudaError_t launch_precond_large(const PrecondArgs<T>& a, int nrhs, cudaStream_t s,
                                 cudaError_t (*zsweeps)(const PrecondArgs<T>&, int, cudaStream_t)) {
    if constexpr (sizeof(T) == 4) {
        if (a.nx == kP128 && a.ny == kP128) {   // on-chip transforms by CTA pairs
            const int sp = large_row_blocks(a.ny);
            dim3 grid(2 * a.nz, nrhs);
            k_fft128_cluster<false, false><<<grid, kP128Threads, kP128Smem, s>>>(a, sp, Fft128Update{});
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = zsweeps(a, nrhs, s);
            if (e != cudaSuccess) return e;
            k_fft128_cluster<true, false><<<grid, kP128Threads, kP128Smem, s>>>(a, sp, Fft128Update{});
            return cudaGetLastError();
        }
    }
    LargeFftArgs<T> f{};
    f.src = a.r;
    f.dst = a.spec;
    f.src_rhs = f.dst_rhs = a.npts;
    f.nx = a.nx;
    f.ny = a.ny;
    f.nz = a.nz;
    f.nf = a.nf;
    f.ax = a.ax;
    f.ay = a.ay;
    f.twx = a.twx;
    f.twy = a.twy;
    f.state = a.state;
    f.mask = a.mask;
    f.npts = a.npts;
    cudaError_t e = launch_rows<T, 0>(f, a.nz, nrhs, s);
    if (e == cudaSuccess)
        e = launch_cols<T>(a.spec, a.npts, a.nz, nrhs, a.nx, a.ny, a.ay, a.twy, 0, a.state, a.mask, s);
    if (e == cudaSuccess) e = zsweeps(a, nrhs, s);
    if (e == cudaSuccess)
        e = launch_cols<T>(a.spec, a.npts, a.nz, nrhs, a.nx, a.ny, a.ay, a.twy, 1, a.state, a.mask, s);
    if (e != cudaSuccess) return e;
    LargeFftArgs<T> g = f;
    g.src = a.spec;
    g.dst = a.z;
    g.inv = 1;
    g.r = a.r;
    g.dot_part = a.dot_part;
    g.nrm_part = a.nrm_part;
    g.slot_stride = a.slot_stride;
    g.slot_base = 0;
    return launch_rows<T, 1>(g, a.nz, nrhs, s);
}

// COCG update x += alpha p, r -= alpha q fused with the forward transform of r, the
// z-sweeps and the inverse transform, for 128 x 128 FP32 planes (the on-chip CTA-pair
// transforms); cudaErrorNotSupported for other planes
cudaError_t launch_update_precond_128(const PrecondArgs<float>& a, int nrhs, cudaStream_t s, float2* x,
                                      float2* r, float2* const* pbufs, const float2* q,
                                      cudaError_t (*zsweeps)(const PrecondArgs<float>&, int, cudaStream_t)) {
    if (a.nx != kP128 || a.ny != kP128) return cudaErrorNotSupported;
    const int sp = large_row_blocks(a.ny);
    dim3 grid(2 * a.nz, nrhs);
    Fft128Update u{x, r, {pbufs[0], pbufs[1]}, q};
    k_fft128_cluster<false, true><<<grid, kP128Threads, kP128Smem, s>>>(a, sp, u);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = zsweeps(a, nrhs, s);
    if (e != cudaSuccess) return e;
    k_fft128_cluster<true, false><<<grid, kP128Threads, kP128Smem, s>>>(a, sp, Fft128Update{});
    return cudaGetLastError();
}

// self-energy through the two-pass transforms; scratch: 2 * nrhs * 2 nf * nxy
// elements; partial slots from slot_base: 2 nf * row blocks
template <typename T>
cudaError_t launch_sigma_large(const SigmaArgs<T>& a, int nrhs, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    const int nxy = a.nx * a.ny;
    const long long cs = 2LL * a.nf * nxy;   // compact stride between RHS
    C* sin = a.scratch;
    C* sout = a.scratch + cs * nrhs;
    LargeFftArgs<T> f{};
    f.src = a.x;
    f.srcp[0] = a.pnew[0];
    f.srcp[1] = a.pnew[1];
    f.dst = sin;
    f.src_rhs = a.npts;
    f.dst_rhs = cs;
    f.src_end = 1;
    f.dst_end = 0;
    f.nx = a.nx;
    f.ny = a.ny;
    f.nz = a.nz;
    f.nf = a.nf;
    f.ax = a.ax;
    f.ay = a.ay;
    f.twx = a.twx;
    f.twy = a.twy;
    f.state = a.state;
    f.mask = a.mask;
    f.npts = a.npts;
    const int np = 2 * a.nf;
    cudaError_t e = launch_rows<T, 0>(f, np, nrhs, s);
    if (e == cudaSuccess) e = launch_cols<T>(sin, cs, np, nrhs, a.nx, a.ny, a.ay, a.twy, 0, a.state, a.mask, s);
    if (e != cudaSuccess) return e;
    dim3 gm((nxy + 255) / 256, 2, nrhs);
    k_sigma_mix_large<T><<<gm, 256, 0, s>>>(sin, sout, a.sigma, a.rhs_energy, nxy, a.nf, a.state, a.mask);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_cols<T>(sout, cs, np, nrhs, a.nx, a.ny, a.ay, a.twy, 1, a.state, a.mask, s);
    if (e != cudaSuccess) return e;
    LargeFftArgs<T> g = f;
    g.src = sout;
    g.srcp[0] = g.srcp[1] = nullptr;
    g.src_rhs = cs;
    g.src_end = 0;
    g.inv = 1;
    g.y = a.y;
    g.xop = a.x;
    g.xopp[0] = a.pnew[0];
    g.xopp[1] = a.pnew[1];
    g.dot_part = a.dot_part;
    g.slot_stride = a.slot_stride;
    g.slot_base = a.slot_base;
    return launch_rows<T, 2>(g, np, nrhs, s);
}

template cudaError_t launch_precond_large<float>(const PrecondArgs<float>&, int, cudaStream_t,
                                                 cudaError_t (*)(const PrecondArgs<float>&, int, cudaStream_t));
template cudaError_t launch_precond_large<double>(const PrecondArgs<double>&, int, cudaStream_t,
                                                  cudaError_t (*)(const PrecondArgs<double>&, int, cudaStream_t));
template cudaError_t launch_sigma_large<float>(const SigmaArgs<float>&, int, cudaStream_t);
template cudaError_t launch_sigma_large<double>(const SigmaArgs<double>&, int, cudaStream_t);

}  // namespace iobm
