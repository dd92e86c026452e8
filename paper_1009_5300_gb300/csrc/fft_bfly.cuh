// The radix butterflies of every lateral FFT of the library (Eq. 19's transform
// in the self-energy, the Fourier preconditioners and the large-plane passes):
// the R-point DFT kernel and the runtime-indexed Stockham butterfly built on it.
// The compile-time plane FFT (fft_ct.cuh) uses the same kernel with constant
// index arithmetic.
#pragma once

#include "iobm_internal.cuh"
#include "complex_ops.cuh"

#include <type_traits>
#include <utility>

namespace iobm {

// f(std::integral_constant<int, k>) for k = 0 .. K-1 (compile-time loop index)
template <int K, typename F, int... I>
__device__ __forceinline__ void ct_for_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int K, typename F>
__device__ __forceinline__ void ct_for(F&& f) {
    ct_for_impl<K>(f, std::make_integer_sequence<int, K>{});
}

// cos and sin on [0, pi/2] by their Taylor series (constant expressions; the terms
// fall below 1e-17 of the sum within 24 terms there)
__host__ __device__ constexpr double ct_series_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 24; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_series_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 24; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}

// cos and sin of 2 pi E / R as compile-time constants: 2 pi E / R = q pi/2 + th with
// the quadrant q and th = (pi/2) rem / R in [0, pi/2)
template <int R, int E>
struct UnitRoot {
    static constexpr int e = ((E % R) + R) % R;
    static constexpr int q = (4 * e) / R;
    static constexpr int rem = 4 * e - q * R;
    static constexpr double th = 1.57079632679489661923132169163975 * rem / R;
    static constexpr double c0 = ct_series_cos(th), s0 = ct_series_sin(th);
    static constexpr double cos = q == 0 ? c0 : (q == 1 ? -s0 : (q == 2 ? -c0 : s0));
    static constexpr double sin = q == 0 ? s0 : (q == 1 ? c0 : (q == 2 ? -s0 : -c0));
};

// v exp(-+2 pi i E / R) (forward: -, inverse: +) with a compile-time exponent: the
// powers 0, R/4, R/2, 3R/4 cost no multiplication
template <typename C, int R, int E, bool INV>
__device__ __forceinline__ C ct_root_mul(C v) {
    constexpr int e = ((E % R) + R) % R;
    C r;
    if constexpr (e == 0) {
        r = v;
    } else if constexpr (2 * e == R) {
        r.x = -v.x; r.y = -v.y;
    } else if constexpr (4 * e == R || 4 * e == 3 * R) {
        // exp(-i pi/2) = -i; exp(+i pi/2) = +i; 3R/4 the opposite
        constexpr bool times_i = (4 * e == R) == INV;
        if constexpr (times_i) { r.x = -v.y; r.y = v.x; } else { r.x = v.y; r.y = -v.x; }
    } else {
        using T = decltype(v.x);
        constexpr T c = (T)UnitRoot<R, e>::cos;
        constexpr T s = (T)(INV ? UnitRoot<R, e>::sin : -UnitRoot<R, e>::sin);
        r.x = v.x * c - v.y * s;
        r.y = v.x * s + v.y * c;
    }
    return r;
}

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

// o = R-point DFT of v held in registers, R in {2, 3, 4, 8, 12, 16}, with the
// direction a compile-time constant.  R = 4A (A = R/4) splits as A DFTs of 4 points
// on v[n1 + A n2], the twiddles exp(-+2 pi i n1 k2 / R), and 4 DFTs of A points:
// o[k2 + 4 k1] = sum_n1 exp(-+2 pi i n1 k1 / A) W^(n1 k2) sum_n2 v[n1 + A n2] exp(-+2 pi i n2 k2 / 4).
template <typename C, int R, bool INV>
__device__ __forceinline__ void dft_reg(const C (&v)[R], C (&o)[R]) {
    if constexpr (R <= 4) {
        small_dft<C, R>(v, o, nullptr, 1, INV);
    } else {
        static_assert(R % 4 == 0 && R / 4 <= 4, "register DFT sizes: 2, 3, 4, 8, 12, 16");
        constexpr int A = R / 4;
        C y[A][4];
        ct_for<A>([&](auto n1c) {
            constexpr int n1 = decltype(n1c)::value;
            C in[4], out[4];
#pragma unroll
            for (int n2 = 0; n2 < 4; ++n2) in[n2] = v[n1 + A * n2];
            small_dft<C, 4>(in, out, nullptr, 1, INV);
            ct_for<4>([&](auto k2c) {
                constexpr int k2 = decltype(k2c)::value;
                y[n1][k2] = ct_root_mul<C, R, n1 * k2, INV>(out[k2]);
            });
        });
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            C in[A], out[A];
#pragma unroll
            for (int n1 = 0; n1 < A; ++n1) in[n1] = y[n1][k2];
            small_dft<C, A>(in, out, nullptr, 1, INV);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) o[k2 + 4 * k1] = out[k1];
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
