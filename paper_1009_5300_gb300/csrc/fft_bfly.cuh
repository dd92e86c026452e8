// The radix butterflies of every lateral FFT of the library (Eq. 19's transform
// in the self-energy, the Fourier preconditioners and the large-plane passes):
// the R-point DFT kernel and the runtime-indexed Stockham butterfly built on it.
// The compile-time plane FFT (fft_ct.cuh) uses the same kernel with constant
// index arithmetic.
#pragma once

#include "iobm_internal.cuh"
#include "complex_ops.cuh"

namespace iobm {

// o_a = sum_b v_b exp(-+2 pi i a b / R) (forward: -, inverse: +).  Radices 2, 4 and 3
// use their closed forms; any other R reads its roots from the N-point twiddle table
// tw[t] = exp(-2 pi i t / N), root a b at tw[((a b) mod R) NR] with NR = N / R.
template <typename C, int R>
__device__ __forceinline__ void small_dft(const C (&v)[R], C (&o)[R], const C* tw, int NR, bool inv) {
    if constexpr (R == 2) {
        o[0] = cadd(v[0], v[1]);
        o[1] = csub(v[0], v[1]);
    } else if constexpr (R == 4) {
        const C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        const C a2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        C a3;   // -i d (forward) or +i d (inverse)
        if (inv) { a3.x = -d.y; a3.y = d.x; } else { a3.x = d.y; a3.y = -d.x; }
        o[0] = cadd(a0, a2);
        o[2] = csub(a0, a2);
        o[1] = cadd(a1, a3);
        o[3] = csub(a1, a3);
    } else if constexpr (R == 3) {
        // exp(-+2 pi i / 3) = -1/2 -+ i sqrt(3)/2
        using T = decltype(v[0].x);
        const T c = (T)-0.5, sn = (T)0.86602540378443864676;
        const C t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
        o[0] = cadd(v[0], t1);
        C m;
        m.x = v[0].x + c * t1.x;
        m.y = v[0].y + c * t1.y;
        C js;   // -i sn t2 (forward) or +i sn t2 (inverse)
        if (inv) { js.x = -sn * t2.y; js.y = sn * t2.x; } else { js.x = sn * t2.y; js.y = -sn * t2.x; }
        o[1] = cadd(m, js);
        o[2] = csub(m, js);
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
}

// Butterfly j of a Stockham pass of radix R over sub-transforms of size Ns of an
// N-point line (runtime N, Ns): v_r = src[(j + r N/R) ss] W^(r (j mod Ns) N/(Ns R)),
// o = R-point DFT of v; output r belongs at index base + r Ns (returned base =
// (j / Ns) Ns R + j mod Ns).
template <typename C, int R>
__device__ __forceinline__ int stockham_bfly_out(const C* src, int ss, int N, int Ns, int j,
                                                 const C* __restrict__ tw, bool inv, C (&o)[R]) {
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
    small_dft<C, R>(v, o, tw, NR, inv);
    return (j / Ns) * Ns * R + k;
}

template <typename C, int R>
__device__ __forceinline__ void stockham_bfly(const C* src, int ss, C* dst, int ds, int N, int Ns,
                                              int j, const C* __restrict__ tw, bool inv) {
    C o[R];
    const int base = stockham_bfly_out<C, R>(src, ss, N, Ns, j, tw, inv, o);
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * Ns) * ds] = o[r];
}

// the same butterfly for the runtime radices 2, 3, 4, 5 of an FftAxis plan
template <typename C>
__device__ __forceinline__ void stockham_bfly_rt(int R, const C* src, int ss, C* dst, int ds, int N,
                                                 int Ns, int j, const C* tw, bool inv) {
    switch (R) {
        case 2: stockham_bfly<C, 2>(src, ss, dst, ds, N, Ns, j, tw, inv); break;
        case 3: stockham_bfly<C, 3>(src, ss, dst, ds, N, Ns, j, tw, inv); break;
        case 4: stockham_bfly<C, 4>(src, ss, dst, ds, N, Ns, j, tw, inv); break;
        case 5: stockham_bfly<C, 5>(src, ss, dst, ds, N, Ns, j, tw, inv); break;
        default: break;   // plans only hold the radices above (checked on the host)
    }
}

}  // namespace iobm
