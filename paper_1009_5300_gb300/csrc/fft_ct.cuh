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
#include "fft_bfly.cuh"

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

// one R-point butterfly j of a pass with compile-time sizes: reads
// src[(j + r N/R) ss], returns the R outputs (small_dft of fft_bfly.cuh) and the
// index of the first (output r goes to base + r NS)
template <typename C, int N, int NS, int R>
__device__ __forceinline__ int ct_bfly_out(const C* src, int ss, int j, const C* tw, bool inv,
                                           C (&o)[R]) {
    constexpr int NR = N / R;
    constexpr int TS = N / (NS * R);
    const int k = j % NS;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        C u = src[(j + r * NR) * ss];
        if (r && NS > 1) {   // the first pass has k = 0: every twiddle is 1
            // r k TS <= (R - 1)(NS - 1) N / (NS R) < N: no reduction mod N needed
            C w = tw[r * k * TS];
            if (inv) w.y = -w.y;
            u = cmul(u, w);
        }
        v[r] = u;
    }
    small_dft<C, R>(v, o, tw, NR, inv);
    return (j / NS) * NS * R + k;
}

template <typename C, int N, int NS, int R>
__device__ __forceinline__ void ct_bfly(const C* src, int ss, C* dst, int ds, int j,
                                        const C* tw, bool inv) {
    C o[R];
    const int base = ct_bfly_out<C, N, NS, R>(src, ss, j, tw, inv, o);
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * NS) * ds] = o[r];
}

// all passes of N-point transforms along N lines (line stride ls, element stride es)
// by a CTA of NT threads
template <typename C, int N, int P, int NS, int NT>
__device__ __forceinline__ void ct_passes(C*& cur, C*& oth, int ls, int es, const C* tw, bool inv) {
    if constexpr (P < CtPlan<N>::npass) {
        constexpr int R = CtPlan<N>::radix(P);
        constexpr int NB = N * (N / R);   // butterflies of the pass
        // line index fastest: a row pass then touches elements line * (N + 1) + c,
        // an odd stride that spreads 16 consecutive lines over 16 different 8-byte
        // bank pairs, and a column pass touches consecutive elements
#pragma unroll
        for (int k = 0; k < (NB + NT - 1) / NT; ++k) {
            const int t = threadIdx.x + k * NT;
            if (NB % NT == 0 || t < NB) {
                const int line = t % N, j = t / N;
                ct_bfly<C, N, NS, R>(cur + line * ls, es, oth + line * ls, es, j, tw, inv);
            }
        }
        __syncthreads();
        C* s = cur; cur = oth; oth = s;
        ct_passes<C, N, P + 1, NS * R, NT>(cur, oth, ls, es, tw, inv);
    }
}

// Row-major element i = tid + K NT of an N x N plane, as its index in the padded
// shared-memory layout (rows of pitch PT), from the thread's first row and column
// (row0, col0) = (tid / N, tid % N): the step K NT is a compile-time constant, so
// only a compare and adds remain.
template <int N, int NT, int PT, int K>
__device__ __forceinline__ int ct_padded_index(int row0, int col0) {
    constexpr int dr = (K * NT) / N, dc = (K * NT) % N;
    const int c = col0 + dc;
    return (c >= N) ? (row0 + dr + 1) * PT + (c - N) : (row0 + dr) * PT + c;
}

// Output positions of the last column pass for a CTA of NT threads: thread tid
// handles butterflies t = tid + k NT (k < K) of column t % N and index
// j = t / N < N / R, whose R outputs are rows j + r N / R; output "slot" k R + r.
template <int N, int NT>
struct CtLastPass {
    static constexpr int R = CtPlan<N>::radix(CtPlan<N>::npass - 1);
    static constexpr int NS = N / R;                  // sub-transform size before the pass
    static constexpr int K = (N * NS + NT - 1) / NT;  // butterflies per thread
    static constexpr int SLOTS = K * R;
    __device__ static bool pos(int tid, int k, int r, int& row, int& col) {
        const int t = tid + k * NT;
        if (t >= N * NS) return false;
        col = t % N;
        row = t / N + r * NS;
        return true;
    }
};

// Column passes of a 2D transform whose last pass hands every output to
// store(row, col, value, slot) (slot as in CtLastPass, a compile-time constant
// after unrolling) instead of writing it back to shared memory; consecutive
// threads store consecutive columns of a row.  The CTA has NT threads.
template <typename C, int N, int P, int NS, int NT, typename Store>
__device__ __forceinline__ void ct_col_passes_store(C*& cur, C*& oth, int pitch, const C* tw,
                                                    bool inv, Store& store) {
    constexpr int R = CtPlan<N>::radix(P);
    constexpr int PER = N / R;
    if constexpr (P + 1 < CtPlan<N>::npass) {
#pragma unroll
        for (int k = 0; k < (N * PER + NT - 1) / NT; ++k) {
            const int t = threadIdx.x + k * NT;
            if ((N * PER) % NT == 0 || t < N * PER) {
                const int line = t % N, j = t / N;
                ct_bfly<C, N, NS, R>(cur + line, pitch, oth + line, pitch, j, tw, inv);
            }
        }
        __syncthreads();
        C* s = cur; cur = oth; oth = s;
        ct_col_passes_store<C, N, P + 1, NS * R, NT>(cur, oth, pitch, tw, inv, store);
    } else {
        constexpr int K = (N * PER + NT - 1) / NT;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int t = threadIdx.x + k * NT;
            if (t < N * PER) {
                const int line = t % N, j = t / N;
                C o[R];
                const int base = ct_bfly_out<C, N, NS, R>(cur + line, pitch, j, tw, inv, o);
#pragma unroll
                for (int r = 0; r < R; ++r) store(base + r * NS, line, o[r], k * R + r);
            }
        }
    }
}

// Shared-memory pitch of a plane row: one element of padding so that the
// column passes (stride = pitch) spread over the banks instead of hitting one.
template <int N> struct CtPitch { static constexpr int P = N + 1; };

// 2D FFT of an N x N plane in shared memory (a, rows of pitch N+1), b scratch of
// the same shape; returns the buffer that holds the result
template <typename C, int N, int NT>
__device__ __forceinline__ C* ct_fft2(C* a, C* b, const C* tw, bool inv) {
    constexpr int P = CtPitch<N>::P;
    C* cur = a;
    C* oth = b;
    ct_passes<C, N, 0, 1, NT>(cur, oth, P, 1, tw, inv);   // rows
    ct_passes<C, N, 0, 1, NT>(cur, oth, 1, P, tw, inv);   // columns
    return cur;
}

// The same transform with the outputs delivered to store(row, col, value) by the
// last column pass (no trailing shared-memory round trip and barrier).
template <typename C, int N, int NT, typename Store>
__device__ __forceinline__ void ct_fft2_store(C* a, C* b, const C* tw, bool inv, Store store) {
    constexpr int P = CtPitch<N>::P;
    C* cur = a;
    C* oth = b;
    ct_passes<C, N, 0, 1, NT>(cur, oth, P, 1, tw, inv);   // rows
    ct_col_passes_store<C, N, 0, 1, NT>(cur, oth, P, tw, inv, store);
}

// Two-factor plan N = R1 R2 for the sizes whose first radix fits in registers: per
// axis, one pass of R1-point DFTs in registers (sub-transform size 1: no twiddles)
// and one pass of R2-point DFTs after the twiddles exp(-+2 pi i r j / N).  A CTA of
// NT = N R2 threads holds one plane; every thread does one R1-point DFT per first
// pass and K2 = R1 / R2 R2-point DFTs per second pass.
template <int N> struct Ct2Plan { static constexpr bool ok = false; };
template <> struct Ct2Plan<32> { static constexpr bool ok = true; static constexpr int R1 = 8, R2 = 4; };
template <> struct Ct2Plan<48> { static constexpr bool ok = true; static constexpr int R1 = 12, R2 = 4; };
template <> struct Ct2Plan<64> { static constexpr bool ok = true; static constexpr int R1 = 16, R2 = 4; };
template <int N>
struct Ct2Shape {
    static constexpr int R1 = Ct2Plan<N>::R1, R2 = Ct2Plan<N>::R2;
    static constexpr int NT = N * R2;
    static constexpr int K2 = R1 / R2;
    static constexpr int PT = N + 1;   // shared-memory row pitch
    static_assert(R1 * R2 == N && R1 % R2 == 0, "two-factor plan");
    // the first pass's inputs of thread tid: row tid / R2, columns tid % R2 + m R2 (m < R1)
    __device__ static int in_row(int tid) { return tid / R2; }
    __device__ static int in_col(int tid, int m) { return tid % R2 + m * R2; }
    // the last pass's outputs of thread tid: column tid % N, rows j + a R1 with
    // j = tid / N + k R2 (k < K2, a < R2), handed to the store as slot k R2 + a
    __device__ static int out_row(int tid, int k, int a) { return tid / N + k * R2 + a * R1; }
    __device__ static int out_col(int tid) { return tid % N; }
};

// 2D transform of one N x N plane by NT threads in one shared-memory plane A (pitch
// N + 1).  v holds the thread's inputs of the first row pass (Ct2Shape::in_row /
// in_col: the caller reads them from global memory), store(row, col, value, slot) takes
// the output from the last column pass.  tw holds exp(-2 pi i t / N), t < N, and must be
// visible to every thread before the first barrier inside.
//
// Pass 1 (rows): thread (row y, j = tid % R2) forms the R1-point DFT of x[y][j + m R2]
// into A[y][j R1 + a]; pass 2 (rows): butterfly (y, j < R1), y fastest, reads
// A[y][j + r R1] exp(-+2 pi i r j / N) and writes its R2-point DFT to the same
// positions (in place: the butterflies touch disjoint sets); pass 3 (columns) reads
// A[j + m R2][x], holds its outputs across a barrier and writes them to rows
// j R1 + a; pass 4 (columns, in place) hands its outputs to the store.  Every
// shared-memory access of a warp touches each 8-byte bank pair at most twice.
template <typename C, int N, bool INV, typename Store>
__device__ __forceinline__ void ct2_fft2(const C (&v1)[Ct2Plan<N>::R1], C* A, const C* tw,
                                         Store store) {
    using S = Ct2Shape<N>;
    constexpr int R1 = S::R1, R2 = S::R2, NT = S::NT, K2 = S::K2, PT = S::PT;
    const int tid = threadIdx.x;
    auto twiddled = [&](C v, int e) {   // v exp(-+2 pi i e / N), 0 <= e < N
        C w = tw[e];
        if (INV) w.y = -w.y;
        return cmul(v, w);
    };
    {   // pass 1: rows, R1 points from the input
        const int j = tid % R2, y = tid / R2;
        C o[R1];
        dft_reg<C, R1, INV>(v1, o);
#pragma unroll
        for (int a = 0; a < R1; ++a) A[y * PT + j * R1 + a] = o[a];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K2; ++k) {   // pass 2: rows, R2 points, in place
        const int t = tid + k * NT;
        const int y = t % N, j = t / N;
        C v[R2], o[R2];
        v[0] = A[y * PT + j];
#pragma unroll
        for (int r = 1; r < R2; ++r) v[r] = twiddled(A[y * PT + j + r * R1], r * j);
        dft_reg<C, R2, INV>(v, o);
#pragma unroll
        for (int a = 0; a < R2; ++a) A[y * PT + j + a * R1] = o[a];
    }
    __syncthreads();
    {   // pass 3: columns, R1 points; every input read before any output is written
        const int x = tid % N, j = tid / N;
        C v[R1], o[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) v[m] = A[(j + m * R2) * PT + x];
        dft_reg<C, R1, INV>(v, o);
        __syncthreads();
#pragma unroll
        for (int a = 0; a < R1; ++a) A[(j * R1 + a) * PT + x] = o[a];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K2; ++k) {   // pass 4: columns, R2 points, to the store
        const int t = tid + k * NT;
        const int x = t % N, j = t / N;
        C v[R2], o[R2];
        v[0] = A[j * PT + x];
#pragma unroll
        for (int r = 1; r < R2; ++r) v[r] = twiddled(A[(j + r * R1) * PT + x], r * j);
        dft_reg<C, R2, INV>(v, o);
#pragma unroll
        for (int a = 0; a < R2; ++a) store(j + a * R1, x, o[a], k * R2 + a);
    }
}

}  // namespace iobm
