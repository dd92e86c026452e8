// Complex FD stencil + V (Eqs. 1-4) on FP64 data in double-float arithmetic.
//
// The FP64 residual r = b - A x of the mixed solver (and its final check) needs
// FP64-class accuracy, not FP64 throughput, and GB300 executes FP64 at a small
// fraction of its FP32 rate.  Every FP64 operand is split exactly into an FP32
// pair hi + lo by integer bit operations (hi: the leading 24 significant bits,
// lo: the remaining bits truncated to 24), the taps are accumulated with
// error-free FP32 transformations (the two-sum of Knuth and the fused
// multiply-add product error), and the result
// is reassembled with one FP64 addition per component.  About 47 significant
// bits are carried through; the relative error is of order 2^-46 of the
// largest term, far below what the FP64 residual check resolves.
//
// Tiling as the register-pipelined FP32 row kernel: a CTA owns kRowTY full
// rows of one RHS for a chunk of z-planes, keeps the z-neighbours of its
// points in a register queue and stages the current plane (own rows plus the
// N_f periodic halo rows above and below, with N_f periodic pad columns) in
// shared memory.  Taps in direct form: diagonal - 2 sum_n c_n, plus
// c_n (x_{+n} + x_{-n}) per axis.
#include "iobm_internal.cuh"
#include "complex_ops.cuh"
#include "dfloat.cuh"

namespace iobm {

constexpr int kDfRowTY = 8;

template <int NF>
__global__ void __launch_bounds__(512) k_stencil_rows_df(const StencilArgs<double> a) {
    extern __shared__ __align__(16) unsigned char smem_df[];
    float4* tile = reinterpret_cast<float4*>(smem_df);   // [SR][TP]: hi.re, hi.im, lo.re, lo.im

    const int rhs = blockIdx.z;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;

    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int TP = nx + 2 * NF;
    const int tid = threadIdx.x;
    const int x = tid % nx;
    const int ly = tid / nx;
    const int ty0 = blockIdx.x * kDfRowTY;
    const int rows = min(kDfRowTY, ny - ty0);
    const bool own = ly < rows;
    const int k0 = blockIdx.y * a.zchunk;
    const int k1 = min(k0 + a.zchunk, nz);
    const long long plane = (long long)nx * ny;
    const long long base = (long long)rhs * a.npts;
    const double2* __restrict__ X = a.x + base;
    double2* __restrict__ Y = a.y + base;
    double tapsum2 = 0.0;
#pragma unroll
    for (int n = 1; n <= NF; ++n) tapsum2 += 2.0 * (a.cx[n] + a.cy[n] + a.cz[n]);
    const double ed = a.ediag ? a.ediag[a.rhs_energy ? a.rhs_energy[rhs] : 0] : 0.0;
    const double cen = a.c0 + ed - tapsum2;   // direct-form diagonal

    // halo rows this thread stages: tile rows ly and ly + kDfRowTY outside the own rows
    constexpr int SR = kDfRowTY + 2 * NF;
    bool hf[2];
    long long hlat[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int srow = ly + t * kDfRowTY;
        hf[t] = srow < 2 * NF + rows && !(srow >= NF && srow < NF + rows) && srow < SR;
        int gy = (ty0 - NF + srow) % ny;
        if (gy < 0) gy += ny;
        hlat[t] = (long long)gy * nx + x;
    }
    const int tcol = NF + x;
    // periodic copy of column x in the pad columns (nx >= NF: at most one... or two
    // when nx < 2 NF)
    const int tpad = (x < NF) ? NF + nx + x : -1;
    const int tpad2 = (x >= nx - NF) ? x - (nx - NF) : -1;
    const long long own_lat = own ? (long long)(ty0 + ly) * nx + x : 0;

    auto raw = [&](int k, long long lat) -> double2 {
        return (k >= 0 && k < nz) ? X[(long long)k * plane + lat] : make_double2(0.0, 0.0);
    };
    Dfc q[2 * NF + 1];
#pragma unroll
    for (int j = 0; j < 2 * NF; ++j) q[j] = df_load(own ? raw(k0 - NF + j, own_lat) : make_double2(0.0, 0.0));
    // loads one plane ahead: own value of plane k+NF, halo of plane k
    double2 onext = own ? raw(k0 + NF, own_lat) : make_double2(0.0, 0.0);
    double2 hnext[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) hnext[t] = hf[t] ? raw(k0, hlat[t]) : make_double2(0.0, 0.0);
    double vnext = (a.V && own) ? a.V[(long long)k0 * plane + own_lat] : 0.0;

    auto put = [&](int srow, const Dfc& v) {
        const float4 f = make_float4(v.hi.x, v.hi.y, v.lo.x, v.lo.y);
        float4* r = tile + srow * TP;
        r[tcol] = f;
        if (tpad >= 0) r[tpad] = f;
        if (tpad2 >= 0) r[tpad2] = f;
    };
    auto get = [&](int idx) -> Dfc {
        const float4 f = tile[idx];
        Dfc r;
        r.hi = make_float2(f.x, f.y);
        r.lo = make_float2(f.z, f.w);
        return r;
    };

    for (int k = k0; k < k1; ++k) {
        q[2 * NF] = df_load(onext);
        Dfc hv[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) hv[t] = df_load(hnext[t]);
        const double vk = vnext;
        // next plane's operands
        onext = (own && k + 1 + NF < nz) ? raw(k + 1 + NF, own_lat) : make_double2(0.0, 0.0);
#pragma unroll
        for (int t = 0; t < 2; ++t)
            hnext[t] = (hf[t] && k + 1 < k1) ? raw(k + 1, hlat[t]) : make_double2(0.0, 0.0);
        if (a.V && own && k + 1 < k1) vnext = a.V[(long long)(k + 1) * plane + own_lat];
        __syncthreads();   // the previous plane's taps are done
#pragma unroll
        for (int t = 0; t < 2; ++t)
            if (hf[t]) put(ly + t * kDfRowTY, hv[t]);
        if (own) put(NF + ly, q[NF]);
        __syncthreads();
        if (own) {
            const double d = a.V ? fma(a.vsign, vk, cen) : cen;
            float dh, dl;
            df_split(d, dh, dl);
            Dfc acc = df_scale(dh, dl, q[NF]);
            const int c = (NF + ly) * TP + tcol;
#pragma unroll
            for (int n = 1; n <= NF; ++n) {
                df_acc(acc, a.dfz[n], df_add(q[NF - n], q[NF + n]));
                df_acc(acc, a.dfx[n], df_add(get(c - n), get(c + n)));
                df_acc(acc, a.dfy[n], df_add(get(c - n * TP), get(c + n * TP)));
            }
            Y[(long long)k * plane + own_lat] =
                make_double2(df_widen(acc.hi.x) + df_widen(acc.lo.x), df_widen(acc.hi.y) + df_widen(acc.lo.y));
        }
#pragma unroll
        for (int j = 0; j < 2 * NF; ++j) q[j] = q[j + 1];
    }
}

bool stencil_df_supported(int nx, int nf) { return nx >= nf && nx >= 4 && nx <= 64; }

cudaError_t launch_stencil_df(const StencilArgs<double>& a0, int nrhs, cudaStream_t s) {
    StencilArgs<double> a = a0;
    if (a.zchunk <= 0) a.zchunk = 32;
    const int tiles_y = (a.ny + kDfRowTY - 1) / kDfRowTY;
    const int nzc = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles_y, nzc, nrhs);
    const int threads = a.nx * kDfRowTY;
    const size_t smem = sizeof(float4) * (size_t)(kDfRowTY + 2 * a.nf) * (a.nx + 2 * a.nf);
    switch (a.nf) {
        case 1: k_stencil_rows_df<1><<<grid, threads, smem, s>>>(a); break;
        case 2: k_stencil_rows_df<2><<<grid, threads, smem, s>>>(a); break;
        case 3: k_stencil_rows_df<3><<<grid, threads, smem, s>>>(a); break;
        case 4: k_stencil_rows_df<4><<<grid, threads, smem, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace iobm
