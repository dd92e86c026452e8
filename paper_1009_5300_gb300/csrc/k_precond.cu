// Lateral-Fourier free-propagator preconditioner
//     z = M r,   M = (E - T - H~)^{-1}
// where T is the FD kinetic operator (Eq. 1) and H~ the jellium self-energy on
// the end planes (Eqs. 7-2, 18-2).  The paper's preconditioner (Eq. 10) is a
// truncated real-space Green's function of the Laplacian meant to approximate
// [E - H_T - H~]^{-1}; here the approximation is the exact Green's function of
// the potential-free transition region, which the lateral Fourier transform of
// Eq. 19 diagonalises: per lateral mode nu it is a banded z-system of
// bandwidth N_f whose LU factors are the same on every plane except the last
// N_f (eliminating a plane of the left lead reproduces the lead), so one
// application costs two plane-FFT passes and one forward/backward z-sweep.
//
// Kernels: (1) forward 2D FFT of every plane of r (one CTA per plane, shared
// memory ping-pong Stockham passes over all lines at once); (2) per-mode
// z-sweeps in place on the spectrum (one thread per mode, coalesced across
// modes); (3) inverse 2D FFT of every plane, fused with the Krylov dot
// products r^T z and |r|^2 of that plane.  The same transforms also apply the
// Eq. 10 preconditioner in its lateral Fourier form (step 2 then being a
// per-mode tridiagonal multiply in z).
#include "iobm_internal.cuh"
#include "complex_ops.cuh"
#include "dfloat.cuh"
#include "fft_bfly.cuh"
#include "fft_ct.cuh"

namespace iobm {

// 2D FFT of an ny x nx plane held in a (x fastest); b is a same-size scratch.
// Every pass spreads the butterflies of all lines over the whole CTA.
// Returns the buffer that holds the result.
template <typename C>
__device__ C* fft2_block(C* a, C* b, const FftAxis& ax, const FftAxis& ay, const C* twx,
                         const C* twy, bool inv) {
    const int nx = ax.n, ny = ay.n;
    C* cur = a;
    C* oth = b;
    int Ns = 1;
    for (int p = 0; p < ax.npass; ++p) {
        const int R = ax.radix[p];
        const int per = nx / R;
        for (int t = threadIdx.x; t < ny * per; t += blockDim.x) {
            const int row = t / per, j = t - row * per;
            stockham_bfly_rt(R, cur + row * nx, 1, oth + row * nx, 1, nx, Ns, j, twx, inv);
        }
        __syncthreads();
        C* s = cur; cur = oth; oth = s;
        Ns *= R;
    }
    Ns = 1;
    for (int p = 0; p < ay.npass; ++p) {
        const int R = ay.radix[p];
        const int per = ny / R;
        for (int t = threadIdx.x; t < nx * per; t += blockDim.x) {
            const int col = t / per, j = t - col * per;
            stockham_bfly_rt(R, cur + col, nx, oth + col, nx, ny, Ns, j, twy, inv);
        }
        __syncthreads();
        C* s = cur; cur = oth; oth = s;
        Ns *= R;
    }
    return cur;
}

template <typename T>
__global__ void __launch_bounds__(256) k_plane_fft_fwd(const PrecondArgs<T> a) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int plane = blockIdx.x, rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    const int nxy = a.nx * a.ny;
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + nxy;
    const long long off = (long long)rhs * a.npts + (long long)plane * nxy;
    for (int i = threadIdx.x; i < nxy; i += blockDim.x) A[i] = a.r[off + i];
    __syncthreads();
    C* res = fft2_block(A, B, a.ax, a.ay, a.twx, a.twy, false);
    for (int i = threadIdx.x; i < nxy; i += blockDim.x) a.spec[off + i] = res[i];
}

// z-sweeps of one lateral mode: forward substitution with the constant band
// multipliers over planes 0 .. nz-nf-1, a dense nf x nf solve on the last nf
// planes, backward substitution with the constant band rows.  In place on the
// spectrum; one thread per (RHS, mode), loads issued kZPrefetch planes ahead.
// In FP32 solves the few modes nearest their channel threshold, whose banded
// z-systems are the worst conditioned, sweep in double-float arithmetic with FP64
// factors (extra blocks at the front of the grid); the others sweep in FP32.
constexpr int kZPrefetch = 8;
constexpr int kZThreads = 128;

template <typename CW, typename CS>
__device__ __forceinline__ CW zcvt(CS v) {
    CW r;
    r.x = v.x;
    r.y = v.y;
    return r;
}

// the sweeps of one mode in working precision CW on storage CS (s: plane 0 of the
// mode, planes nxy apart; pc: the mode's kPcStrideDev factors)
template <typename CW, typename CS, int NF>
__device__ __forceinline__ void zsweep(CS* __restrict__ s, const CW* __restrict__ pc, int nz, int nxy) {
    using W = decltype(CW{}.x);
    CW l[NF + 1], u[NF + 1];
#pragma unroll
    for (int j = 1; j <= NF; ++j) l[j] = pc[j - 1];
#pragma unroll
    for (int j = 0; j <= NF; ++j) u[j] = pc[NF + j];
    const CW uinv = cdivc(make_one<CW>(), u[0]);
    const int m = nz - NF;
    const W scale = (W)1 / (W)nxy;   // the forward FFT carries no 1/N_xy
    constexpr int PF = kZPrefetch;
    // forward: y_k = r_k - sum_j l_j y_{k-j}
    CW hist[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) hist[j] = czero<CW>();   // hist[j] = y_{k-1-j}
    CW buf[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j) buf[j] = (j < m) ? zcvt<CW>(s[(long long)j * nxy]) : czero<CW>();
    for (int k0 = 0; k0 < m; k0 += PF) {
        CW cur[PF];
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            cur[j] = buf[j];
            const int kk = k0 + PF + j;
            buf[j] = (kk < m) ? zcvt<CW>(s[(long long)kk * nxy]) : czero<CW>();
        }
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int k = k0 + j;
            if (k < m) {
                // the newest term last: the older ones do not wait for y_{k-1}
                CW y = cscale(cur[j], scale);
#pragma unroll
                for (int t = NF; t >= 1; --t) y = csub(y, cmul(l[t], hist[t - 1]));
                s[(long long)k * nxy] = zcvt<CS>(y);
#pragma unroll
                for (int t = NF - 1; t > 0; --t) hist[t] = hist[t - 1];
                hist[0] = y;
            }
        }
    }
    // last nf planes: g_i = r_i - sum_{j: i-j < m} l_j y_{i-j};  x_2 = S2^{-1} g
    CW g[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        CW v = cscale(zcvt<CW>(s[(long long)(m + i) * nxy]), scale);
#pragma unroll
        for (int j = 1; j <= NF; ++j)
            if (j > i) v = csub(v, cmul(l[j], hist[j - 1 - i]));
        g[i] = v;
    }
    CW nxt[NF];   // nxt[j] = x_{k+1+j}
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        CW v = czero<CW>();
        // the end block's inverse is read here, where it is used
#pragma unroll
        for (int j = 0; j < NF; ++j) v = cfma(pc[2 * NF + 1 + i * NF + j], g[j], v);
        s[(long long)(m + i) * nxy] = zcvt<CS>(v);
        nxt[i] = v;
    }
    // backward: x_k = (y_k - sum_j u_j x_{k+j}) / u_0
#pragma unroll
    for (int j = 0; j < PF; ++j)
        buf[j] = (m - 1 - j >= 0) ? zcvt<CW>(s[(long long)(m - 1 - j) * nxy]) : czero<CW>();
    for (int k0 = m - 1; k0 >= 0; k0 -= PF) {
        CW cur[PF];
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            cur[j] = buf[j];
            const int kk = k0 - PF - j;
            buf[j] = (kk >= 0) ? zcvt<CW>(s[(long long)kk * nxy]) : czero<CW>();
        }
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int k = k0 - j;
            if (k >= 0) {
                CW v = cur[j];
#pragma unroll
                for (int t = NF; t >= 1; --t) v = csub(v, cmul(u[t], nxt[t - 1]));
                v = cmul(v, uinv);
                s[(long long)k * nxy] = zcvt<CS>(v);
#pragma unroll
                for (int t = NF - 1; t > 0; --t) nxt[t] = nxt[t - 1];
                nxt[0] = v;
            }
        }
    }
}

// The same sweeps in double-float arithmetic (about 47 bits) on FP32 storage, with
// FP64 factors split into FP32 pairs: the forward and backward recurrences carry
// the double-float values; the spectrum between them is stored in FP32.
__device__ __forceinline__ Dfc df_neg(Dfc a) {
    a.hi.x = -a.hi.x; a.hi.y = -a.hi.y; a.lo.x = -a.lo.x; a.lo.y = -a.lo.y;
    return a;
}

template <int NF>
__device__ __forceinline__ void zsweep_df(float2* __restrict__ s, const double2* __restrict__ pc,
                                          int nz, int nxy) {
    // forward factors -l_j; backward factors -u_j / u_0 and 1 / u_0 (formed in FP64 once)
    Dfc nl[NF + 1], nw[NF + 1];
#pragma unroll
    for (int j = 1; j <= NF; ++j) nl[j] = df_neg(df_load(pc[j - 1]));
    const double2 u0 = pc[NF];
    const double den = u0.x * u0.x + u0.y * u0.y;
    const double2 ui = make_double2(u0.x / den, -u0.y / den);
    const Dfc uinv = df_load(ui);
#pragma unroll
    for (int j = 1; j <= NF; ++j) {
        const double2 uj = pc[NF + j];
        nw[j] = df_load(make_double2(-(uj.x * ui.x - uj.y * ui.y), -(uj.x * ui.y + uj.y * ui.x)));
    }
    float sch, scl;
    df_split(1.0 / (double)nxy, sch, scl);   // the forward FFT carries no 1/N_xy
    const Dfc zero = df_from(make_float2(0.f, 0.f));
    const int m = nz - NF;
    constexpr int PF = kZPrefetch;
    Dfc hist[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) hist[j] = zero;
    float2 buf[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j) buf[j] = (j < m) ? s[(long long)j * nxy] : make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < m; k0 += PF) {
        float2 cur[PF];
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            cur[j] = buf[j];
            const int kk = k0 + PF + j;
            buf[j] = (kk < m) ? s[(long long)kk * nxy] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int k = k0 + j;
            if (k < m) {
                // the newest term last: the older ones do not wait for y_{k-1}
                Dfc y = df_scale(sch, scl, df_from(cur[j]));
#pragma unroll
                for (int t = NF; t >= 1; --t) df_cacc(y, nl[t], hist[t - 1]);
                df_norm(y);
                s[(long long)k * nxy] = df_round(y);
#pragma unroll
                for (int t = NF - 1; t > 0; --t) hist[t] = hist[t - 1];
                hist[0] = y;
            }
        }
    }
    Dfc g[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        Dfc v = df_scale(sch, scl, df_from(s[(long long)(m + i) * nxy]));
#pragma unroll
        for (int j = 1; j <= NF; ++j)
            if (j > i) df_cacc(v, nl[j], hist[j - 1 - i]);
        df_norm(v);
        g[i] = v;
    }
    Dfc nxt[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        Dfc v = zero;
#pragma unroll
        for (int j = 0; j < NF; ++j) df_cacc(v, df_load(pc[2 * NF + 1 + i * NF + j]), g[j]);
        df_norm(v);
        s[(long long)(m + i) * nxy] = df_round(v);
        nxt[i] = v;
    }
#pragma unroll
    for (int j = 0; j < PF; ++j)
        buf[j] = (m - 1 - j >= 0) ? s[(long long)(m - 1 - j) * nxy] : make_float2(0.f, 0.f);
    for (int k0 = m - 1; k0 >= 0; k0 -= PF) {
        float2 cur[PF];
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            cur[j] = buf[j];
            const int kk = k0 - PF - j;
            buf[j] = (kk >= 0) ? s[(long long)kk * nxy] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < PF; ++j) {
            const int k = k0 - j;
            if (k >= 0) {
                // x_k = y_k / u_0 - sum_t (u_t / u_0) x_{k+t}, the newest term last
                Dfc x = zero;
                df_cacc(x, uinv, df_from(cur[j]));
#pragma unroll
                for (int t = NF; t >= 1; --t) df_cacc(x, nw[t], nxt[t - 1]);
                df_norm(x);
                s[(long long)k * nxy] = df_round(x);
#pragma unroll
                for (int t = NF - 1; t > 0; --t) nxt[t] = nxt[t - 1];
                nxt[0] = x;
            }
        }
    }
}

// The same sweeps split along z into S segments, one lane each (a group of kZfLanes
// lanes per (RHS, mode)).  The interior recurrences have constant coefficients, so a
// segment's true values are its particular solution from a zero history plus the
// responses to the true history at its start: y_{k0+j} = y^_{k0+j} + sum_i T_i(j) y_{k0-1-i},
// T_i the response to a unit history value (tabulated per mode in FP64, stored as
// float pairs).  Phase 1: every lane solves its segment from a zero history; phase 2:
// the S - 1 segment starts are chained lane to lane by shuffles (each a N_f x N_f
// multiply-add); phase 3: every lane adds its correction.  The backward sweep likewise
// from the top, its first history being the end block's values.  The serial chain per
// sweep falls from m planes to about 2 m / S planes plus S carry steps.
constexpr int kZfLanes = 8;

__device__ __forceinline__ Dfc df_from4(float4 v) {
    Dfc r;
    r.hi = make_float2(v.x, v.y);
    r.lo = make_float2(v.z, v.w);
    return r;
}
__device__ __forceinline__ float4 df_to4(const Dfc& a) { return make_float4(a.hi.x, a.hi.y, a.lo.x, a.lo.y); }
// the previous lane's value within the group of kZfLanes lanes
__device__ __forceinline__ Dfc df_shfl_up(const Dfc& v, unsigned gm) {
    Dfc r;
    r.hi.x = __shfl_up_sync(gm, v.hi.x, 1, kZfLanes);
    r.hi.y = __shfl_up_sync(gm, v.hi.y, 1, kZfLanes);
    r.lo.x = __shfl_up_sync(gm, v.lo.x, 1, kZfLanes);
    r.lo.y = __shfl_up_sync(gm, v.lo.y, 1, kZfLanes);
    return r;
}
__device__ __forceinline__ Dfc df_shfl(const Dfc& v, int src, unsigned gm) {
    Dfc r;
    r.hi.x = __shfl_sync(gm, v.hi.x, src, kZfLanes);
    r.hi.y = __shfl_sync(gm, v.hi.y, src, kZfLanes);
    r.lo.x = __shfl_sync(gm, v.lo.x, src, kZfLanes);
    r.lo.y = __shfl_sync(gm, v.lo.y, src, kZfLanes);
    return r;
}

template <int NF>
__device__ __forceinline__ void zsweep_df_seg(float2* __restrict__ s, const double2* __restrict__ pc,
                                              const float4* __restrict__ tab, float4* __restrict__ scr,
                                              int nz, int nxy, int S, int L, int Lt, int sig, unsigned gm) {
    Dfc nl[NF + 1], nw[NF + 1];
#pragma unroll
    for (int j = 1; j <= NF; ++j) nl[j] = df_neg(df_load(pc[j - 1]));
    const double2 u0 = pc[NF];
    const double den = u0.x * u0.x + u0.y * u0.y;
    const double2 ui = make_double2(u0.x / den, -u0.y / den);
    const Dfc uinv = df_load(ui);
#pragma unroll
    for (int j = 1; j <= NF; ++j) {
        const double2 uj = pc[NF + j];
        nw[j] = df_load(make_double2(-(uj.x * ui.x - uj.y * ui.y), -(uj.x * ui.y + uj.y * ui.x)));
    }
    float sch, scl;
    df_split(1.0 / (double)nxy, sch, scl);   // the forward FFT carries no 1/N_xy
    const Dfc zero = df_from(make_float2(0.f, 0.f));
    const int m = nz - NF;
    const float4* __restrict__ tf = tab;             // [NF][Lt] forward responses
    const float4* __restrict__ tb = tab + NF * Lt;   // backward
    const bool act = sig < S;
    // the next segment's history from this one's tail and its own history C
    auto chain = [&](const float4* t, const Dfc (&tail)[NF], Dfc (&C)[NF]) {
        for (int step = 1; step < S; ++step) {
            Dfc cand[NF];
#pragma unroll
            for (int i = 0; i < NF; ++i) {
                cand[i] = tail[i];
#pragma unroll
                for (int i2 = 0; i2 < NF; ++i2) df_cacc(cand[i], df_from4(t[i2 * Lt + (L - 1 - i)]), C[i2]);
                df_norm(cand[i]);
            }
#pragma unroll
            for (int i = 0; i < NF; ++i) {
                const Dfc up = df_shfl_up(cand[i], gm);
                if (sig == step) C[i] = up;
            }
        }
    };

    // ---- forward: y_k = r_k / N_xy - sum_t l_t y_{k-t}, segment [lo, hi)
    const int lo = sig * L, hi = (sig == S - 1) ? m : lo + L;
    Dfc hist[NF];   // hist[i] = y^_{k-1-i}
#pragma unroll
    for (int i = 0; i < NF; ++i) hist[i] = zero;
    if (act)
        for (int k = lo; k < hi; ++k) {
            Dfc y = df_scale(sch, scl, df_from(s[(long long)k * nxy]));
#pragma unroll
            for (int t = NF; t >= 1; --t) df_cacc(y, nl[t], hist[t - 1]);
            df_norm(y);
            scr[k] = df_to4(y);
#pragma unroll
            for (int t = NF - 1; t > 0; --t) hist[t] = hist[t - 1];
            hist[0] = y;
        }
    Dfc C[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) C[i] = zero;
    chain(tf, hist, C);
    if (act)
        for (int k = lo; k < hi; ++k) {
            Dfc y = df_from4(scr[k]);
#pragma unroll
            for (int i = 0; i < NF; ++i) df_cacc(y, df_from4(tf[i * Lt + (k - lo)]), C[i]);
            df_norm(y);
            s[(long long)k * nxy] = df_round(y);
#pragma unroll
            for (int t = NF - 1; t > 0; --t) hist[t] = hist[t - 1];
            hist[0] = y;   // the last segment ends with the true y_{m-1-i}
        }
    // ---- the last nf planes (every lane, from the last segment's values)
    Dfc yl[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) yl[i] = df_shfl(hist[i], S - 1, gm);
    Dfc g[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        Dfc v = df_scale(sch, scl, df_from(s[(long long)(m + i) * nxy]));
#pragma unroll
        for (int j = 1; j <= NF; ++j)
            if (j > i) df_cacc(v, nl[j], yl[j - 1 - i]);
        df_norm(v);
        g[i] = v;
    }
    Dfc xe[NF];   // x_{m+i}
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        Dfc v = zero;
#pragma unroll
        for (int j = 0; j < NF; ++j) df_cacc(v, df_load(pc[2 * NF + 1 + i * NF + j]), g[j]);
        df_norm(v);
        xe[i] = v;
    }
    __syncwarp(gm);   // every lane read the last planes' r and every segment stored its y
    if (sig == 0)
#pragma unroll
        for (int i = 0; i < NF; ++i) s[(long long)(m + i) * nxy] = df_round(xe[i]);

    // ---- backward: x_k = y_k / u_0 - sum_t (u_t / u_0) x_{k+t}, segment [bot, top)
    const int top = m - sig * L, bot = (sig == S - 1) ? 0 : top - L;
    Dfc nxt[NF];   // nxt[i] = x^_{k+1+i}
#pragma unroll
    for (int i = 0; i < NF; ++i) nxt[i] = zero;
    if (act)
        for (int k = top - 1; k >= bot; --k) {
            Dfc x = zero;
            df_cacc(x, uinv, df_from(s[(long long)k * nxy]));
#pragma unroll
            for (int t = NF; t >= 1; --t) df_cacc(x, nw[t], nxt[t - 1]);
            df_norm(x);
            scr[k] = df_to4(x);
#pragma unroll
            for (int t = NF - 1; t > 0; --t) nxt[t] = nxt[t - 1];
            nxt[0] = x;   // at the end nxt[i] = x^_{bot+i}
        }
#pragma unroll
    for (int i = 0; i < NF; ++i) C[i] = (sig == 0) ? xe[i] : zero;   // x_{top+i} of segment 0
    chain(tb, nxt, C);
    if (act)
        for (int k = top - 1; k >= bot; --k) {
            Dfc x = df_from4(scr[k]);
#pragma unroll
            for (int i = 0; i < NF; ++i) df_cacc(x, df_from4(tb[i * Lt + (top - 1 - k)]), C[i]);
            df_norm(x);
            s[(long long)k * nxy] = df_round(x);
        }
}

// every mode but the double-float ones (flagged in zflag), in the working precision
template <typename T, int NF>
__global__ void __launch_bounds__(kZThreads) k_zsolve(const PrecondArgs<T> a) {
    using C = typename Cplx<T>::type;
    const int rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    const int nxy = a.nx * a.ny;
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= nxy) return;
    const int e = a.rhs_energy ? a.rhs_energy[rhs] : 0;
    if (sizeof(T) == 4 && a.zf_k > 0 && a.zflag[(size_t)e * nxy + mode]) return;
    zsweep<C, C, NF>(a.spec + (long long)rhs * a.npts + mode,
                     a.pc + ((size_t)e * nxy + mode) * kPcStrideDev, a.nz, nxy);
}

// the double-float sweeps of the flagged modes (FP32 solves; beside or before k_zsolve):
// with segments a group of kZfLanes lanes per (RHS, mode), else one thread
template <int NF>
__global__ void __launch_bounds__(kZThreads) k_zsolve_df(const PrecondArgs<float> a) {
    const int rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = a.rhs_energy ? a.rhs_energy[rhs] : 0;
    if (a.zf_S > 1) {
        const int f = t / kZfLanes;
        if (f >= a.zf_k) return;   // the lanes of a group leave together
        const int sig = t % kZfLanes;
        const unsigned gm = ((1u << kZfLanes) - 1u) << (threadIdx.x & 31 & ~(kZfLanes - 1));
        const int mode = a.zf_bins[(size_t)e * a.zf_k + f];
        const int m = a.nz - NF;
        zsweep_df_seg<NF>(a.spec + (long long)rhs * a.npts + mode,
                          a.zf_pc + ((size_t)e * a.zf_k + f) * kPcStrideDev,
                          a.zf_tab + ((size_t)e * a.zf_k + f) * 2 * NF * a.zf_Lt,
                          a.zf_scr + ((size_t)rhs * a.zf_k + f) * m, a.nz, a.nx * a.ny, a.zf_S,
                          a.zf_L, a.zf_Lt, sig, gm);
        return;
    }
    const int f = t;
    if (f >= a.zf_k) return;
    const int mode = a.zf_bins[(size_t)e * a.zf_k + f];
    zsweep_df<NF>(a.spec + (long long)rhs * a.npts + mode,
                  a.zf_pc + ((size_t)e * a.zf_k + f) * kPcStrideDev, a.nz, a.nx * a.ny);
}

// Eq. 10 in the lateral Fourier basis: with r~ the (unnormalised) plane
// spectrum of mode (kx, ky), z~(k) = (1 + 2 C_1 (cos th_x + cos th_y)) r~(k)
//   + C_1 (r~(k-1) + r~(k+1)), th = 2 pi k / N, zero beyond the end planes.
// One thread per (RHS, mode), in place: r~(k+1) is read before z~(k) is written
// and r~(k-1) is kept in a register.  Carries the 1/N_xy of the transform pair.
template <typename T>
__global__ void __launch_bounds__(kZThreads) k_zmul_eq10(const PrecondArgs<T> a) {
    using C = typename Cplx<T>::type;
    const int rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    const int nxy = a.nx * a.ny;
    const int mode = blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= nxy) return;
    const int kx = mode % a.nx, ky = mode / a.nx;
    const double pi2 = 6.283185307179586476925286766559;
    const double d = 1.0 + 2.0 * a.c1 * (cos(pi2 * kx / a.nx) + cos(pi2 * ky / a.ny));
    const T scale = (T)1 / (T)nxy;
    const T dd = (T)d * scale, cc = (T)a.c1 * scale;
    C* __restrict__ s = a.spec + (long long)rhs * a.npts + mode;
    C prev = czero<C>();
    C cur = s[0];
    for (int k = 0; k < a.nz; ++k) {
        const C next = (k + 1 < a.nz) ? s[(long long)(k + 1) * nxy] : czero<C>();
        s[(long long)k * nxy] = caxpy(cc, cadd(prev, next), cscale(cur, dd));
        prev = cur;
        cur = next;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_plane_ifft_dots(const PrecondArgs<T> a) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3 * 8];
    const int plane = blockIdx.x, rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    const int nxy = a.nx * a.ny;
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + nxy;
    const long long off = (long long)rhs * a.npts + (long long)plane * nxy;
    for (int i = threadIdx.x; i < nxy; i += blockDim.x) A[i] = a.spec[off + i];
    __syncthreads();
    C* res = fft2_block(A, B, a.ax, a.ay, a.twx, a.twy, true);
    T dre = 0, dim = 0, nrm = 0;
    for (int i = threadIdx.x; i < nxy; i += blockDim.x) {
        const C z = res[i];
        a.z[off + i] = z;
        if (a.dot_part) {
            const C r = a.r[off + i];
            dre += r.x * z.x - r.y * z.y;
            dim += r.x * z.y + r.y * z.x;
            nrm += r.x * r.x + r.y * r.y;
        }
    }
    if (a.dot_part) {
        double d0 = dre, d1 = dim, d2 = nrm;
        block_reduce_3(d0, d1, d2, red);
        if (threadIdx.x == 0) {
            a.dot_part[(long long)rhs * a.slot_stride + plane] = make_double2(d0, d1);
            a.nrm_part[(long long)rhs * a.slot_stride + plane] = d2;
        }
    }
}

// x += alpha p, r -= alpha q for one plane (COCG update), then the forward FFT
// of the new r into the spectrum buffer.  With alpha_from_state = 0 it is the
// plain forward transform of r.
template <typename T, int N>
__global__ void __launch_bounds__(256, 4) k_update_fft_ct(const PrecondArgs<T> a, typename Cplx<T>::type* x,
                                                       typename Cplx<T>::type* r_rw,
                                                       typename Cplx<T>::type* p0,
                                                       typename Cplx<T>::type* p1,
                                                       const typename Cplx<T>::type* q, int update) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int plane = blockIdx.x, rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    constexpr int NXY = N * N;
    constexpr int PT = CtPitch<N>::P;
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + N * PT;
    C* tw = B + N * PT;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.twx[i];
    const long long off = (long long)rhs * a.npts + (long long)plane * NXY;
    if (update) {
        const C al = from_d2<C>(a.state[rhs].alpha);
        const C* __restrict__ P = ((a.state[rhs].pbuf & 1) ? p1 : p0) + off;
        C* __restrict__ Xv = x + off;
        C* __restrict__ R = r_rw + off;
        const C* __restrict__ Q = q + off;
        // all loads of this thread's points first, then the arithmetic and stores
        constexpr int PER = (NXY + 255) / 256;
        C rv[PER], qv[PER], xv[PER], pv[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int i = threadIdx.x + j * 256;
            if (i < NXY) {
                rv[j] = R[i];
                qv[j] = Q[i];
                xv[j] = Xv[i];
                pv[j] = P[i];
            }
        }
        const int row0 = threadIdx.x / N, col0 = threadIdx.x % N;
        ct_for<PER>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const int i = threadIdx.x + j * 256;
            if (NXY % 256 == 0 || i < NXY) {
                const C rn = csub(rv[j], cmul(al, qv[j]));
                R[i] = rn;
                A[ct_padded_index<N, 256, PT, j>(row0, col0)] = rn;
                Xv[i] = cfma(al, pv[j], xv[j]);
            }
        });
    } else {
        for (int i = threadIdx.x; i < NXY; i += blockDim.x) A[(i / N) * PT + (i % N)] = a.r[off + i];
    }
    __syncthreads();
    C* __restrict__ spec = a.spec + off;
    ct_fft2_store<C, N, 256>(A, B, tw, false,
                             [&](int row, int col, C v, int) { spec[row * N + col] = v; });
}

// CTAs of 256 threads per SM that the shared memory of a plane transform
// (two padded N x N planes and the twiddles) allows, at most 5
template <typename T, int N>
struct CtOccupancy {
    static constexpr int kSmem = (int)sizeof(typename Cplx<T>::type) * (2 * N * (N + 1) + N) + 1024;
    static constexpr int kFit = (227 * 1024) / kSmem;
    static constexpr int value = kFit < 1 ? 1 : (kFit > 5 ? 5 : kFit);
};

template <typename T, int N>
__global__ void __launch_bounds__(256, (CtOccupancy<T, N>::value)) k_ifft_dots_ct(const PrecondArgs<T> a) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3 * 8];
    const int plane = blockIdx.x, rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    constexpr int NXY = N * N;
    constexpr int PT = CtPitch<N>::P;
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + N * PT;
    C* tw = B + N * PT;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.twx[i];
    const long long off = (long long)rhs * a.npts + (long long)plane * NXY;
    {
        constexpr int PER = (NXY + 255) / 256;
        const int row0 = threadIdx.x / N, col0 = threadIdx.x % N;
        ct_for<PER>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const int i = threadIdx.x + j * 256;
            if (NXY % 256 == 0 || i < NXY) A[ct_padded_index<N, 256, PT, j>(row0, col0)] = a.spec[off + i];
        });
    }
    // r at the positions this thread's last column pass produces, loaded now so
    // the loads overlap the transform
    using L = CtLastPass<N, 256>;
    C* __restrict__ zo = a.z + off;
    const C* __restrict__ rin = a.r + off;
    const bool dots = a.dot_part != nullptr;
    C rv[L::SLOTS];
#pragma unroll
    for (int k = 0; k < L::K; ++k)
#pragma unroll
        for (int r = 0; r < L::R; ++r) {
            int row, col;
            rv[k * L::R + r] = (dots && L::pos(threadIdx.x, k, r, row, col)) ? rin[row * N + col] : czero<C>();
        }
    __syncthreads();
    // the last column pass stores z and forms r^T z and |r|^2 on the way
    T dre = 0, dim = 0, nrm = 0;
    ct_fft2_store<C, N, 256>(A, B, tw, true, [&](int row, int col, C z, int slot) {
        zo[row * N + col] = z;
        if (dots) {
            const C r = rv[slot];
            dre += r.x * z.x - r.y * z.y;
            dim += r.x * z.y + r.y * z.x;
            nrm += r.x * r.x + r.y * r.y;
        }
    });
    if (a.dot_part) {
        double d0 = dre, d1 = dim, d2 = nrm;
        block_reduce_3(d0, d1, d2, red);
        if (threadIdx.x == 0) {
            a.dot_part[(long long)rhs * a.slot_stride + plane] = make_double2(d0, d1);
            a.nrm_part[(long long)rhs * a.slot_stride + plane] = d2;
        }
    }
}

// The same inverse transform and dot products on the two-factor plan (N = 32, 48,
// 64): the first row pass reads the spectrum from global memory, the last column
// pass writes z, so a point crosses shared memory twice per axis; r at the outputs
// of the thread's last pass is loaded with the spectrum, so its latency overlaps
// the transform.  One shared-memory plane per CTA (the passes work in place); CTAs of
// N R2 threads (192 at N = 48), at most five per SM (three at N = 64; FP64: two), which
// the registers of the prefetched operands allow without spills.
template <typename T, int N>
struct Ct2Occupancy {
    static constexpr size_t kDyn = sizeof(typename Cplx<T>::type) * ((size_t)N * (N + 1) + N);
    static constexpr int kSmem = (int)kDyn + 1024 + 192;
    static constexpr int kFit = (228 * 1024) / kSmem;
    static constexpr int kCap = sizeof(typename Cplx<T>::type) == 8 ? (N >= 64 ? 3 : 5) : 2;
    static constexpr int value = kFit < 1 ? 1 : (kFit > kCap ? kCap : kFit);
};

template <typename T, int N>
__global__ void __launch_bounds__(Ct2Shape<N>::NT, (Ct2Occupancy<T, N>::value))
    k_ifft2_dots(const PrecondArgs<T> a) {
    using C = typename Cplx<T>::type;
    using S = Ct2Shape<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3 * 8];
    const int plane = blockIdx.x, rhs = blockIdx.y;
    if (a.state && !((1 << a.state[rhs].status) & a.mask)) return;
    constexpr int PT = S::PT;
    C* A = reinterpret_cast<C*>(smem_raw);
    C* tw = A + N * PT;
    for (int i = threadIdx.x; i < N; i += S::NT) tw[i] = a.twx[i];
    const long long off = (long long)rhs * a.npts + (long long)plane * (N * N);
    const C* __restrict__ spec = a.spec + off;
    C* __restrict__ zo = a.z + off;
    const C* __restrict__ rin = a.r + off;
    const bool dots = a.dot_part != nullptr;
    C v[S::R1];
#pragma unroll
    for (int m = 0; m < S::R1; ++m) v[m] = spec[S::in_row(threadIdx.x) * N + S::in_col(threadIdx.x, m)];
    C rv[S::K2 * S::R2];
#pragma unroll
    for (int k = 0; k < S::K2; ++k)
#pragma unroll
        for (int aa = 0; aa < S::R2; ++aa)
            rv[k * S::R2 + aa] = dots ? rin[S::out_row(threadIdx.x, k, aa) * N + S::out_col(threadIdx.x)] : czero<C>();
    T dre = 0, dim = 0, nrm = 0;
    ct2_fft2<C, N, true>(v, A, tw, [&](int row, int col, C z, int slot) {
        zo[row * N + col] = z;
        if (dots) {
            const C r = rv[slot];
            dre += r.x * z.x - r.y * z.y;
            dim += r.x * z.y + r.y * z.x;
            nrm += r.x * r.x + r.y * r.y;
        }
    });
    if (dots) {
        double d0 = dre, d1 = dim, d2 = nrm;
        block_reduce_3(d0, d1, d2, red);
        if (threadIdx.x == 0) {
            a.dot_part[(long long)rhs * a.slot_stride + plane] = make_double2(d0, d1);
            a.nrm_part[(long long)rhs * a.slot_stride + plane] = d2;
        }
    }
}

template <typename T>
size_t precond_smem_bytes(int nx, int ny) {
    using C = typename Cplx<T>::type;
    return 2 * sizeof(C) * (size_t)nx * ny;
}

constexpr int kPrecondSmemLimit = 160 * 1024;

template <typename T>
static cudaError_t prepare_type() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kPrecondSmemLimit);
    };
    set((const void*)k_plane_fft_fwd<T>);
    set((const void*)k_plane_ifft_dots<T>);
#define IOBM_CT(N)                                    \
    set((const void*)k_update_fft_ct<T, N>);          \
    set((const void*)k_ifft_dots_ct<T, N>);
    IOBM_CT(12) IOBM_CT(16) IOBM_CT(24) IOBM_CT(32) IOBM_CT(48) IOBM_CT(64)
#undef IOBM_CT
    set((const void*)k_ifft2_dots<T, 32>);
    set((const void*)k_ifft2_dots<T, 48>);
    set((const void*)k_ifft2_dots<T, 64>);
    return e;
}

cudaError_t precond_prepare() {
    cudaError_t e = prepare_type<float>();
    if (e == cudaSuccess) e = prepare_type<double>();
    return e;
}

static bool ct_size(int nx, int ny) {
    return nx == ny && (nx == 12 || nx == 16 || nx == 24 || nx == 32 || nx == 48 || nx == 64);
}

template <typename T>
static cudaError_t launch_zsolve(const PrecondArgs<T>& a, int nrhs, cudaStream_t s) {
    const int nxy = a.nx * a.ny;
    if (a.eq10) {
        dim3 gz((nxy + kZThreads - 1) / kZThreads, nrhs);
        k_zmul_eq10<T><<<gz, kZThreads, 0, s>>>(a);
        return cudaGetLastError();
    }
    const int nzb = (nxy + kZThreads - 1) / kZThreads;
    if (a.nf < 1 || a.nf > 4) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    const bool fork = sizeof(T) == 4 && a.zf_k > 0 && a.zf_side;
    if (sizeof(T) == 4 && a.zf_k > 0) {
        // the double-float sweeps: on the side stream, forked from s and joined back
        // after the other sweeps, or (no side stream) on s before them
        cudaStream_t sd = s;
        if (fork) {
            e = cudaEventRecord(a.zf_fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(a.zf_side, a.zf_fork, 0);
            if (e != cudaSuccess) return e;
            sd = a.zf_side;
        }
        if constexpr (sizeof(T) == 4) {
            const int per = a.zf_S > 1 ? kZfLanes * a.zf_k : a.zf_k;
            dim3 gd((per + kZThreads - 1) / kZThreads, nrhs);
            switch (a.nf) {
                case 1: k_zsolve_df<1><<<gd, kZThreads, 0, sd>>>(a); break;
                case 2: k_zsolve_df<2><<<gd, kZThreads, 0, sd>>>(a); break;
                case 3: k_zsolve_df<3><<<gd, kZThreads, 0, sd>>>(a); break;
                default: k_zsolve_df<4><<<gd, kZThreads, 0, sd>>>(a); break;
            }
        }
        e = cudaGetLastError();
        if (e == cudaSuccess && fork) e = cudaEventRecord(a.zf_join, sd);
        if (e != cudaSuccess) return e;
    }
    dim3 gz(nzb, nrhs);
    switch (a.nf) {
        case 1: k_zsolve<T, 1><<<gz, kZThreads, 0, s>>>(a); break;
        case 2: k_zsolve<T, 2><<<gz, kZThreads, 0, s>>>(a); break;
        case 3: k_zsolve<T, 3><<<gz, kZThreads, 0, s>>>(a); break;
        default: k_zsolve<T, 4><<<gz, kZThreads, 0, s>>>(a); break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess && fork) e = cudaStreamWaitEvent(s, a.zf_join, 0);
    return e;
}

// forward transform (optionally fused with the COCG update) for square planes
template <typename T>
static cudaError_t launch_fwd_ct(const PrecondArgs<T>& a, int nrhs, cudaStream_t s,
                                 typename Cplx<T>::type* x, typename Cplx<T>::type* r,
                                 typename Cplx<T>::type* p0, typename Cplx<T>::type* p1,
                                 const typename Cplx<T>::type* q, int update) {
    using C = typename Cplx<T>::type;
    const int N = a.nx;
    const size_t smem = sizeof(C) * (2 * (size_t)N * (N + 1) + N);
    dim3 gp(a.nz, nrhs);
    switch (N) {
#define IOBM_CT(NN) \
        case NN: k_update_fft_ct<T, NN><<<gp, 256, smem, s>>>(a, x, r, p0, p1, q, update); break;
        IOBM_CT(12) IOBM_CT(16) IOBM_CT(24) IOBM_CT(32) IOBM_CT(48) IOBM_CT(64)
#undef IOBM_CT
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_inv_ct(const PrecondArgs<T>& a, int nrhs, cudaStream_t s) {
    using C = typename Cplx<T>::type;
    const int N = a.nx;
    const size_t smem = sizeof(C) * (2 * (size_t)N * (N + 1) + N);
    dim3 gp(a.nz, nrhs);
    switch (N) {
#define IOBM_CT(NN) case NN: k_ifft_dots_ct<T, NN><<<gp, 256, smem, s>>>(a); break;
#define IOBM_CT2(NN) \
        case NN: k_ifft2_dots<T, NN><<<gp, Ct2Shape<NN>::NT, Ct2Occupancy<T, NN>::kDyn, s>>>(a); break;
        IOBM_CT(12) IOBM_CT(16) IOBM_CT(24) IOBM_CT2(32) IOBM_CT2(48) IOBM_CT2(64)
#undef IOBM_CT
#undef IOBM_CT2
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_precond_fourier(const PrecondArgs<T>& a, int nrhs, cudaStream_t s) {
    if (a.nx * a.ny > kSmemPlaneLimit) return launch_precond_large<T>(a, nrhs, s, launch_zsolve<T>);
    const size_t smem = precond_smem_bytes<T>(a.nx, a.ny);
    if (smem > (size_t)kPrecondSmemLimit) return cudaErrorInvalidValue;
    cudaError_t e;
    dim3 gp(a.nz, nrhs);
    const bool ct = ct_size(a.nx, a.ny);
    if (ct) {
        e = launch_fwd_ct<T>(a, nrhs, s, nullptr, nullptr, nullptr, nullptr, nullptr, 0);
    } else {
        k_plane_fft_fwd<T><<<gp, 256, smem, s>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    e = launch_zsolve<T>(a, nrhs, s);
    if (e != cudaSuccess) return e;
    if (ct) return launch_inv_ct<T>(a, nrhs, s);
    k_plane_ifft_dots<T><<<gp, 256, smem, s>>>(a);
    return cudaGetLastError();
}

// COCG update x += alpha p, r -= alpha q fused with the preconditioner's forward
// transform of r (square planes with a compile-time plan); returns
// cudaErrorNotSupported when the size has no fused kernel (the caller then
// runs the separate update and launch_precond_fourier).
template <typename T>
cudaError_t launch_update_precond_fourier(const PrecondArgs<T>& a, int nrhs, cudaStream_t s,
                                          typename Cplx<T>::type* x, typename Cplx<T>::type* r,
                                          typename Cplx<T>::type* const* pbufs,
                                          const typename Cplx<T>::type* q,
                                          const cudaEvent_t* ev, int timed) {
    if (!ct_size(a.nx, a.ny)) {
        if constexpr (sizeof(T) == 4)
            return launch_update_precond_128(a, nrhs, s, x, r, pbufs, q, launch_zsolve<float>);
        return cudaErrorNotSupported;
    }
    // event record nodes when captured into a graph
    auto mark = [&](int stage, int k) {
        return (ev && timed == stage) ? cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal)
                                      : cudaSuccess;
    };
    cudaError_t e = mark(1, 0);
    if (e == cudaSuccess) e = launch_fwd_ct<T>(a, nrhs, s, x, r, pbufs[0], pbufs[1], q, 1);
    if (e == cudaSuccess) e = mark(1, 1);
    if (e == cudaSuccess) e = mark(2, 0);
    if (e == cudaSuccess) e = launch_zsolve<T>(a, nrhs, s);
    if (e == cudaSuccess) e = mark(2, 1);
    if (e == cudaSuccess) e = mark(3, 0);
    if (e == cudaSuccess) e = launch_inv_ct<T>(a, nrhs, s);
    if (e == cudaSuccess) e = mark(3, 1);
    return e;
}

template cudaError_t launch_update_precond_fourier<float>(const PrecondArgs<float>&, int, cudaStream_t,
                                                          float2*, float2*, float2* const*,
                                                          const float2*, const cudaEvent_t*, int);
template cudaError_t launch_update_precond_fourier<double>(const PrecondArgs<double>&, int,
                                                           cudaStream_t, double2*, double2*,
                                                           double2* const*, const double2*,
                                                           const cudaEvent_t*, int);

template size_t precond_smem_bytes<float>(int, int);
template size_t precond_smem_bytes<double>(int, int);
template cudaError_t launch_precond_fourier<float>(const PrecondArgs<float>&, int, cudaStream_t);
template cudaError_t launch_precond_fourier<double>(const PrecondArgs<double>&, int, cudaStream_t);

}  // namespace iobm
