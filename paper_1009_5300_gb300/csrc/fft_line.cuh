// Mixed-radix Stockham FFT of one line held in shared memory, by one warp
// (runtime radix plan of radices 2, 3, 4, 5; Eq. 19's lateral transform for
// plane sizes without a compile-time plan).  The butterflies are those of
// fft_bfly.cuh.
#pragma once

#include "iobm_internal.cuh"
#include "complex_ops.cuh"
#include "fft_bfly.cuh"

namespace iobm {

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
        // Stockham pass of radix R: the warp's lanes take butterflies j < N / R
        for (int j = lane; j < N / R; j += 32) stockham_bfly_rt(R, src, ss, dst, ds, N, Ns, j, tw, inv);
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
