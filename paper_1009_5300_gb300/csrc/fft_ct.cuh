// Compile-time Stockham FFT of square N x N planes held in shared memory
// (Eq. 19's lateral transform), shared by the preconditioner and the
// self-energy kernels.  The radix sequence (4s, then 2s, 3s, 5s), the
// sub-transform sizes and every index divisor are constants, so the butterfly
// index arithmetic reduces to multiplies and shifts; every pass spreads the
// butterflies of all N lines over the whole CTA.  The transform is
// unnormalised; the inverse uses the conjugate twiddles.
#pragma once

#include "iobm_internal.cuh"
#include "complex_ops.cuh"

namespace iobm {

// Radix sequence of an N-point transform.  Twiddles (tw[t] = exp(-2 pi i t / N))
// come from a shared-memory copy of the table.
template <int N>
struct CtPlan {
    __host__ __device__ static constexpr int count(int n, int r) {
        return n % r == 0 ? 1 + count(n / r, r) : 0;
    }
    static constexpr int n4 = count(N, 4);
    static constexpr int n2 = count(N / (n4 == 0 ? 1 : (1 << (2 * n4))), 2);
    static constexpr int rest2 = N / (1 << (2 * n4)) / (1 << n2);
    static constexpr int n3 = count(rest2, 3);
    static constexpr int rest3 = rest2 / (n3 == 0 ? 1 : (n3 == 1 ? 3 : (n3 == 2 ? 9 : 27)));
    static constexpr int n5 = count(rest3, 5);
    static constexpr int npass = n4 + n2 + n3 + n5;
    __host__ __device__ static constexpr int radix(int p) {
        return p < n4 ? 4 : (p < n4 + n2 ? 2 : (p < n4 + n2 + n3 ? 3 : 5));
    }
};

template <typename C, int N, int NS, int R>
__device__ __forceinline__ void ct_bfly(const C* src, int ss, C* dst, int ds, int j,
                                        const C* tw, bool inv) {
    constexpr int NR = N / R;
    constexpr int TS = N / (NS * R);
    const int k = j % NS;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        C u = src[(j + r * NR) * ss];
        if (r) {
            C w = tw[(r * k * TS) % N];
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
    const int base = (j / NS) * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * NS) * ds] = o[r];
}

// all passes of N-point transforms along `lines` lines (line stride ls, element stride es)
template <typename C, int N, int P, int NS>
__device__ __forceinline__ void ct_passes(C*& cur, C*& oth, int ls, int es, const C* tw, bool inv) {
    if constexpr (P < CtPlan<N>::npass) {
        constexpr int R = CtPlan<N>::radix(P);
        constexpr int PER = N / R;
        for (int t = threadIdx.x; t < N * PER; t += blockDim.x) {
            const int line = t / PER, j = t - line * PER;
            ct_bfly<C, N, NS, R>(cur + line * ls, es, oth + line * ls, es, j, tw, inv);
        }
        __syncthreads();
        C* s = cur; cur = oth; oth = s;
        ct_passes<C, N, P + 1, NS * R>(cur, oth, ls, es, tw, inv);
    }
}

// Shared-memory pitch of a plane row: one element of padding so that the
// column passes (stride = pitch) spread over the banks instead of hitting one.
template <int N> struct CtPitch { static constexpr int P = N + 1; };

// 2D FFT of an N x N plane in shared memory (a, rows of pitch N+1), b scratch of
// the same shape; returns the buffer that holds the result
template <typename C, int N>
__device__ __forceinline__ C* ct_fft2(C* a, C* b, const C* tw, bool inv) {
    constexpr int P = CtPitch<N>::P;
    C* cur = a;
    C* oth = b;
    ct_passes<C, N, 0, 1>(cur, oth, P, 1, tw, inv);   // rows
    ct_passes<C, N, 0, 1>(cur, oth, 1, P, tw, inv);   // columns
    return cur;
}

}  // namespace iobm
