// Small complex helpers for float2 / double2 (interleaved re, im).
#pragma once
#include <cuda_runtime.h>

namespace iobm {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// Packed two-lane FP32 arithmetic (add/sub/mul/fma.rn.f32x2, one instruction for
// both components of a complex float2)
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
    return ((unsigned long long)__float_as_uint(a.y) << 32) | __float_as_uint(a.x);
}
__device__ __forceinline__ float2 bits_f2(unsigned long long v) {
    return make_float2(__uint_as_float((unsigned)(v & 0xffffffffull)), __uint_as_float((unsigned)(v >> 32)));
}
__device__ __forceinline__ float2 p2add(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(d);
}
__device__ __forceinline__ float2 p2sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(d);
}
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(d);
}
// a * b + c lane-wise
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return bits_f2(d);
}

// a + s * b with real s
__device__ __forceinline__ float2 caxpy(float s, float2 b, float2 a) {
    return make_float2(fmaf(s, b.x, a.x), fmaf(s, b.y, a.y));
}
__device__ __forceinline__ double2 caxpy(double s, double2 b, double2 a) {
    return make_double2(fma(s, b.x, a.x), fma(s, b.y, a.y));
}
// a + b * c (complex)
__device__ __forceinline__ float2 cfma(float2 b, float2 c, float2 a) {
    return make_float2(fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x)), fmaf(b.x, c.y, fmaf(b.y, c.x, a.y)));
}
__device__ __forceinline__ double2 cfma(double2 b, double2 c, double2 a) {
    return make_double2(fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y)));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

template <typename C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

template <typename C> __device__ __forceinline__ C from_d2(double2 v);
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) {
    return make_float2((float)v.x, (float)v.y);
}
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }

template <typename C> __device__ __forceinline__ C make_one();
template <> __device__ __forceinline__ float2 make_one<float2>() { return make_float2(1.f, 0.f); }
template <> __device__ __forceinline__ double2 make_one<double2>() { return make_double2(1.0, 0.0); }

__device__ __forceinline__ float2 cdivc(float2 a, float2 b) {
    const float den = b.x * b.x + b.y * b.y;
    return make_float2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ double2 cdivc(double2 a, double2 b) {
    const double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }

// Deterministic block reduction of (double2 dot, double nrm): fixed tree.
// `red` must hold 3 * (blockDim / 32) doubles.  Result valid in thread 0.
__device__ __forceinline__ void block_reduce_3(double& a, double& b, double& c, double* red) {
    const int lane = threadIdx.x & 31;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int wid = tid >> 5;
    const int lane2 = tid & 31;
    (void)lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int nw = (nthreads + 31) >> 5;
    if (lane2 == 0) {
        red[wid] = a;
        red[nw + wid] = b;
        red[2 * nw + wid] = c;
    }
    __syncthreads();
    if (tid == 0) {
        double sa = 0, sb = 0, sc = 0;
        for (int w = 0; w < nw; ++w) {
            sa += red[w];
            sb += red[nw + w];
            sc += red[2 * nw + w];
        }
        a = sa;
        b = sb;
        c = sc;
    }
}

}  // namespace iobm
