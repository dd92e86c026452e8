// Mixed-radix Stockham FFT of one line held in shared memory, by one warp
// (runtime radix plan of radices 2, 3, 4, 5; Eq. 19's lateral transform for
// plane sizes without a compile-time plan).
#pragma once

#include "iobm_internal.cuh"
#include "complex_ops.cuh"

namespace iobm {

// Stockham mixed-radix FFT of one line held in shared memory, by one warp.
// Pass with radix R over current sub-transform size Ns: for j < N/R,
//   v_r = src[j + r N/R] * W^(r * (j mod Ns) * N/(Ns R)),  W = exp(-+2 pi i / N)
//   out = R-point DFT of v
//   dst[(j / Ns) Ns R + (j mod Ns) + r Ns] = out_r
// followed by a swap of src and dst.
template <typename C, int R>
__device__ __forceinline__ void radix_pass(const C* src, int ss, C* dst, int ds, int N, int Ns,
                                           const C* __restrict__ tw, bool inv, int lane) {
    const int NR = N / R;
    const int tscale = N / (Ns * R);
    for (int j = lane; j < NR; j += 32) {
        const int k = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C u = src[(j + r * NR) * ss];
            const int t = (r * k * tscale) % N;
            C w = tw[t];
            if (inv) w.y = -w.y;
            v[r] = (r == 0) ? u : cmul(u, w);
        }
        C o[R];
        if constexpr (R == 2) {
            o[0] = cadd(v[0], v[1]);
            o[1] = csub(v[0], v[1]);
        } else if constexpr (R == 4) {
            C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
            C a2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
            // a3 = -i d (forward) or +i d (inverse)
            C a3;
            if (inv) { a3.x = -d.y; a3.y = d.x; } else { a3.x = d.y; a3.y = -d.x; }
            o[0] = cadd(a0, a2);
            o[2] = csub(a0, a2);
            o[1] = cadd(a1, a3);
            o[3] = csub(a1, a3);
        } else {
            // generic R-point DFT, roots exp(-+2 pi i a b / R) = tw[(a b mod R) N/R]
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
}

template <typename C>
__device__ void fft_line(C* data, int stride, C* scratch, const FftAxis& ax,
                         const C* __restrict__ tw, bool inv, int lane) {
    const int N = ax.n;
    C* src = data;
    int ss = stride;
    C* dst = scratch;
    int ds = 1;
    int Ns = 1;
    for (int p = 0; p < ax.npass; ++p) {
        const int R = ax.radix[p];
        switch (R) {
            case 2: radix_pass<C, 2>(src, ss, dst, ds, N, Ns, tw, inv, lane); break;
            case 3: radix_pass<C, 3>(src, ss, dst, ds, N, Ns, tw, inv, lane); break;
            case 4: radix_pass<C, 4>(src, ss, dst, ds, N, Ns, tw, inv, lane); break;
            case 5: radix_pass<C, 5>(src, ss, dst, ds, N, Ns, tw, inv, lane); break;
            default: break;   // plans only hold the radices above (checked on the host)
        }
        __syncwarp();
        C* t = src; src = dst; dst = t;
        int tt = ss; ss = ds; ds = tt;
        Ns *= R;
    }
    if (src != data) {
        for (int i = lane; i < N; i += 32) data[i * stride] = src[i];
        __syncwarp();
    }
}

}  // namespace iobm
