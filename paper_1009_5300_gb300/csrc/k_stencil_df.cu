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

namespace iobm {

constexpr int kDfRowTY = 8;

// x = hi + lo: hi the leading 24 significant bits of x (truncated), lo the next
// 24 of the remaining 29 (truncated).  |x| < 2^-100 gives 0, and the lo part is
// dropped below 2^-74; |x| must stay below 2^127.
__device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ffull) - 1023;
    if (e < -100) {
        hi = 0.f;
        lo = 0.f;
        return;
    }
    hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffull));
    const unsigned rem = (unsigned)(b & 0x1fffffffull);
    lo = 0.f;
    if (rem != 0u && e >= -74) {
        const int p = 31 - __clz(rem);   // leading one of the remainder, 0 .. 28
        const unsigned mant = (p >= 23) ? (rem >> (p - 23)) : (rem << (23 - p));
        lo = __uint_as_float(sgn | ((unsigned)(e - 52 + p + 127) << 23) | (mant & 0x7fffffu));
    }
}

// exact float -> double widening by bit operations (zero and subnormals -> 0)
__device__ __forceinline__ double df_widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xffu;
    if (ef == 0u) return 0.0;
    const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned long long e64 = (ef == 0xffu) ? 0x7ffull : (unsigned long long)(ef - 127u + 1023u);
    return __longlong_as_double((long long)(sgn | (e64 << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

struct Dfc {        // complex double-float, lanes (re, im)
    float2 hi, lo;
};

__device__ __forceinline__ Dfc df_load(double2 v) {
    Dfc r;
    df_split(v.x, r.hi.x, r.lo.x);
    df_split(v.y, r.hi.y, r.lo.y);
    return r;
}

// The error-free transformations below use the _rn intrinsics, which the
// compiler never contracts into fused multiply-adds: a product fused into a
// later sum would turn the two-sum's correction into the product's rounding
// error and count it twice.

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// one lane of a + b, unnormalised (the rounding error of hi + hi goes into lo)
__device__ __forceinline__ void df_add1(float ah, float al, float bh, float bl, float& sh, float& sl) {
    float e;
    sh = two_sum(ah, bh, e);
    sl = __fadd_rn(e, __fadd_rn(al, bl));
}

__device__ __forceinline__ Dfc df_add(const Dfc& a, const Dfc& b) {
    Dfc r;
    df_add1(a.hi.x, a.lo.x, b.hi.x, b.lo.x, r.hi.x, r.lo.x);
    df_add1(a.hi.y, a.lo.y, b.hi.y, b.lo.y, r.hi.y, r.lo.y);
    return r;
}

// one lane of acc + c s, c = ch + cl
__device__ __forceinline__ void df_acc1(float& ah, float& al, float ch, float cl, float sh, float sl) {
    const float p = __fmul_rn(ch, sh);
    float e1 = __fmaf_rn(ch, sh, -p);   // the product's rounding error, exactly
    e1 = __fmaf_rn(ch, sl, e1);
    e1 = __fmaf_rn(cl, sh, e1);
    float e2;
    ah = two_sum(ah, p, e2);
    al = __fadd_rn(al, __fadd_rn(e1, e2));
}

// acc + c s for a real double-float weight c = (ch, cl)
__device__ __forceinline__ void df_acc(Dfc& acc, float2 c, const Dfc& s) {
    df_acc1(acc.hi.x, acc.lo.x, c.x, c.y, s.hi.x, s.lo.x);
    df_acc1(acc.hi.y, acc.lo.y, c.x, c.y, s.hi.y, s.lo.y);
}

// acc = d x for a real double-float d = (dh, dl)
__device__ __forceinline__ Dfc df_scale(float dh, float dl, const Dfc& x) {
    Dfc r;
    r.hi.x = __fmul_rn(dh, x.hi.x);
    r.hi.y = __fmul_rn(dh, x.hi.y);
    r.lo.x = __fmaf_rn(dl, x.hi.x, __fmaf_rn(dh, x.lo.x, __fmaf_rn(dh, x.hi.x, -r.hi.x)));
    r.lo.y = __fmaf_rn(dl, x.hi.y, __fmaf_rn(dh, x.lo.y, __fmaf_rn(dh, x.hi.y, -r.hi.y)));
    return r;
}

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
