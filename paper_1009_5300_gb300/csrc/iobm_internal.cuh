// Internal declarations shared by the IOBM CUDA translation units.
//
// Device data layout (all in HBM, one junction per handle):
//   vectors      [rhs][z][y][x] interleaved complex (float2 / double2)
//   V            [z][y][x] real (float and double copies)
//   sigma table  [energy][ky][kx][d][d'] complex, lateral FFT-bin order
//   partials     [rhs][slot] FP64 partial sums of the Krylov dot products
//   scalars      [rhs] RhsState (alpha, beta, rho, norms, status, counters)
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace iobm {

constexpr int kMaxNf = 4;          // FD half-width supported by the kernels
constexpr int kMaxRadixPasses = 12;
constexpr int kMaxRadix = 5;

// ---- per-RHS solver status (device) ---------------------------------
enum RhsStatusCode : int {
    ST_ACTIVE = 0,        // iterating
    ST_PENDING = 1,       // recurrence residual fell: FP64 residual replacement due
    ST_RESTART = 2,       // residual replaced, z/rho must be recomputed
    ST_CONVERGED = 3,
    ST_NOCONV = 4,
    ST_BREAKDOWN = 5,
    ST_IDLE = 6,          // slot not used
};

// status masks selecting which RHS a launch works on
enum : int {
    M_ACTIVE = 1 << ST_ACTIVE,
    M_PENDING = 1 << ST_PENDING,
    M_RESTART = 1 << ST_RESTART,
    M_ALL = 0x7fffffff,
};

struct RhsState {
    double2 rho;        // r^T z of the current iterate
    double2 rho_prev;   // previous r^T z (for beta)
    double2 alpha;
    double2 beta;
    double rr;          // ||r||^2 (recurrence)
    double rr_ref;      // ||r||^2 at the last residual replacement
    double bb;          // ||b||^2
    double res64;       // last FP64 relative residual
    int status;
    int iters;
    int replacements;
    int first;          // 1: next direction update uses beta = 0
    int pbuf;           // which of the two direction buffers holds the current p
    int pad;
};

// Lateral profile of a source: f(l) for b(l, d) = coef[d] * f(l).
enum Profile : int {
    PROF_EXP_PLUS = 0,    // exp(+i G.r)
    PROF_COS = 1,         // cos(G.r)
    PROF_SIN = 2,         // sin(G.r)
    PROF_EXP_MINUS = 3,   // exp(-i G.r)
};

// Source / functional descriptor of one RHS: on the N_f planes of one end
// (depth d), b(l, d) = coef[d] * f(l) with f one of the profiles above.
struct RhsDesc {
    int energy;
    int kx, ky;           // FFT bins of the lateral mode (nu mod N)
    int side;             // planes: 0 -> plane d, 1 -> plane nz-1-d
    int profile;
    int pad;
    double2 coef[kMaxNf];
};



// Lateral FFT plan of one axis
struct FftAxis {
    int n;
    int npass;
    int radix[kMaxRadixPasses];
};

// ---- kernel parameter blocks -------------------------------------------

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename T>
struct StencilArgs {
    using C = typename Cplx<T>::type;
    const C* x;            // operand (COCG: z, with p = z + beta p_old)
    C* pbufs[2];           // COCG: direction buffers; reads p_old = pbufs[pbuf] and
                           // writes p = pbufs[1 - pbuf] (pbuf from the RHS state)
    C* y;                  // result
    const T* V;            // potential or nullptr
    int nx, ny, nz;
    int nf;                // taps per side (1 for the preconditioner)
    T cx[kMaxNf + 1];      // coefficients of x-shifts +-n (index n >= 1)
    T cy[kMaxNf + 1];
    T cz[kMaxNf + 1];
    T c0;                  // centre coefficient + 2 sum of the tap weights (taps are
                           // applied as c_n (x_{+n} + x_{-n} - 2 x_0))
    int iso;               // 1: cx[n] == cy[n] == cz[n] for every n (cubic grid spacing)
    T vsign;               // centre += vsign * V(r)
    const double* ediag;   // per-RHS additive centre term (energy) or nullptr
    const int* rhs_energy; // RHS -> energy index (for ediag)
    const RhsState* state; // status / beta
    int mask;              // process RHS whose status bit is in mask
    int fused_p;           // 1: x is z and p = z + beta*pold is formed and stored
    int dot_mode;          // 0 none, 1: slots += x^T y (and |x|^2 to nrm)
    double2* dot_part;     // [rhs][slot_stride]
    double* nrm_part;      // [rhs][slot_stride] or nullptr
    int slot_stride;
    int slot_base;
    int zchunk;            // planes per CTA
    int tiles_x, tiles_y;  // lateral tiling
    long long npts;
    int* err;              // set to a nonzero code when a bounded wait gives up (or nullptr)
    int variant;           // 0: the fastest kernel for the shape, 1: the register-pipelined row
                           // kernel, 2 (FP64 data): double-float arithmetic, 3: the bulk-copy
                           // row kernel with one row per thread (FP32), 4: the bulk-copy
                           // kernel with a shared-memory ring of operand planes (FP32)
    float2 dfx[kMaxNf + 1];  // variant 2: cx[n], cy[n], cz[n] as FP32 pairs (hi, lo)
    float2 dfy[kMaxNf + 1];
    float2 dfz[kMaxNf + 1];
    long long wait_cycles;   // limit of the bounded copy waits (0: about one second)
    int wait_inject;         // 1: each CTA of the bulk-copy kernel also waits once on a
                             // barrier that no copy completes (tests the give-up path)
    // Lateral Bloch vector kappa in the gauge phi = exp(-i kappa.r) psi (FP64 kernels
    // only): with rhs_sign set, RHS i applies the operator at s kappa, s = rhs_sign[i]
    // = +1 or -1, whose lateral taps are c_n (exp(i s n theta) x_{+n} + exp(-i s n theta)
    // x_{-n}) = bc[n] (x_{+n} + x_{-n}) + i s bs[n] (x_{+n} - x_{-n}), theta = kappa h.
    const int* rhs_sign;
    T bxc[kMaxNf + 1], bxs[kMaxNf + 1];   // c_x,n cos(n kappa_x h_x), c_x,n sin(n kappa_x h_x)
    T byc[kMaxNf + 1], bys[kMaxNf + 1];
};

// the double-float row kernel (FP64 data, operator apply without fused p or dots)
bool stencil_df_supported(int nx, int nf);
cudaError_t launch_stencil_df(const StencilArgs<double>& a, int nrhs, cudaStream_t s);

// codes written to StencilArgs::err
enum { ERR_STAGE_TIMEOUT = 1 };

// Self-energy (boundary) application, one cluster of nf CTAs per (rhs, end)
template <typename T>
struct SigmaArgs {
    using C = typename Cplx<T>::type;
    const C* x;             // operand planes are read from here
    const C* pnew[2];       // if set: operand = pnew[1 - pbuf] of the RHS (COCG direction)
    C* y;                   // y[end planes] -= Sigma x
    C* yend;                // if set (planes <= 4096 points): yend[((rhs 2 + end) nf + d) nxy + i]
                            // = -(Sigma x) of that plane instead, y untouched
    const C* sigma;         // [energy][ky][kx][nf][nf]
    const int* rhs_energy;
    const RhsState* state;
    int mask;
    int nx, ny, nz, nf;
    FftAxis ax, ay;
    const C* twx;           // [nx] exp(-2 pi i k / nx)
    const C* twy;           // [ny]
    double2* dot_part;      // slot_base + end*nf + d (planes > 4096 points: see k_fft_large.cu)
    int slot_stride, slot_base;
    long long npts;
    C* scratch;             // planes > 4096 points: 2 * nrhs * 2 nf * nxy elements
};

template <typename T>
struct KbArgs {
    using C = typename Cplx<T>::type;
    const C* x;
    const C* pnew[2];        // if set: operand = pnew[1 - pbuf] of the RHS (COCG direction)
    const C* zsrc;           // if set: y -= V_NL zsrc, the dot partial still pairs the operand
                             // above with the added term (the implicit operator form)
    C* y;                    // y[support] -= V_NL x
    int nproj;
    const int* pptr;         // [nproj+1] projector CSR
    const int* pidx;
    const T* pval;
    const double* coupling;  // E_p
    double dvol;
    int nunion;
    const int* uidx;         // union of supports (sorted grid indices)
    const int* uptr;         // [nunion+1]
    const int* uproj;        // projector of each entry
    const T* uval;           // value of each entry
    const RhsState* state;
    int mask;
    double2* dot_part;       // one partial per application CTA: slots slot_base + [0, kb_slots)
    int slot_stride, slot_base;
    long long npts;
    C* sp;                   // scratch [rhs][nproj]: E_p dvol <p|x>
    const int* uplane;       // [nz+1]: union points of plane k are uidx[uplane[k] .. uplane[k+1])
    // Lateral Bloch vector (gauge phi = exp(-i kappa.r) psi): with rhs_sign set, the
    // projector of RHS i is p(r) exp(i s kappa.r) on the right and p(r) exp(-i s kappa.r)
    // on the left, s = rhs_sign[i]; gph[l] = exp(i kappa.r_l) on the lateral plane.
    const int* rhs_sign;
    const C* gph;
    int nxy;
};

// dot-product partial slots the KB application writes per RHS
int kb_slots(int nunion);

constexpr int kPcStrideDev = 25;   // per-mode preconditioner table stride (nf = 4)

template <typename T>
struct PrecondArgs {
    using C = typename Cplx<T>::type;
    const C* r;              // operand
    C* spec;                 // spectrum scratch (may alias z)
    C* z;                    // result
    const C* pc;             // [energy][ky][kx][kPcStrideDev]
    const int* rhs_energy;
    const RhsState* state;
    int mask;
    int nx, ny, nz, nf;
    FftAxis ax, ay;
    const C* twx;
    const C* twy;
    double2* dot_part;       // slot = plane
    double* nrm_part;
    int slot_stride;
    long long npts;
    // FP32 solves: per energy slot the zf_k lateral modes nearest their channel
    // threshold take their z-sweeps in FP64, with FP64 factors: zflag[e][bin] = 1 for
    // them, zf_bins[e][f] their bins, zf_pc[e][f][kPcStrideDev] their factors
    const unsigned char* zflag;
    const int* zf_bins;
    const double2* zf_pc;
    int zf_k;
    // the double-float sweeps split z into zf_S segments of zf_L planes (the last one
    // longer, < zf_L + nf), one lane each: zf_tab[e][f][2][nf][zf_Lt] the responses of the
    // forward and backward recurrences to each unit history value (hi.re, hi.im, lo.re,
    // lo.im), zf_scr[rhs][f][nz - nf] the segments' particular solutions
    const float4* zf_tab;
    float4* zf_scr;
    int zf_S, zf_L, zf_Lt;
    // host side: with zf_side set, the double-float sweeps run on stream zf_side
    // (forked from and joined back to the launching stream by the two events)
    // concurrently with the FP32 sweeps of the other modes
    cudaStream_t zf_side;
    cudaEvent_t zf_fork, zf_join;
    int eq10;                // 0: free-propagator z-sweeps (pc tables); 1: Eq. 10 per mode
    double c1;               // Eq. 10 weight exp(-alpha) (eq10 = 1)
};

template <typename T> cudaError_t launch_precond_fourier(const PrecondArgs<T>& a, int nrhs, cudaStream_t s);
// ev (optional): a pair of events recorded around stage `timed` (1 the update +
// forward FFT, 2 the z-sweeps, 3 the inverse FFT + dots)
template <typename T>
cudaError_t launch_update_precond_fourier(const PrecondArgs<T>& a, int nrhs, cudaStream_t s,
                                          typename Cplx<T>::type* x, typename Cplx<T>::type* r,
                                          typename Cplx<T>::type* const* pbufs,
                                          const typename Cplx<T>::type* q,
                                          const cudaEvent_t* ev = nullptr, int timed = 0);
template <typename T> size_t precond_smem_bytes(int nx, int ny);
cudaError_t precond_prepare();
cudaError_t stencil_prepare();

// lateral planes above 4096 points (up to 256 x 256): two-pass global-memory FFTs
constexpr int kSmemPlaneLimit = 4096;
cudaError_t fft_large_prepare();
int large_row_blocks(int ny);
bool large_plane_supported(int nx, int ny);
template <typename T>
cudaError_t launch_precond_large(const PrecondArgs<T>& a, int nrhs, cudaStream_t s,
                                 cudaError_t (*zsweeps)(const PrecondArgs<T>&, int, cudaStream_t));
// update + forward transform + z-sweeps + inverse transform for 128 x 128 FP32 planes
// (on-chip CTA-pair transforms; k_fft_large.cu); cudaErrorNotSupported otherwise
cudaError_t launch_update_precond_128(const PrecondArgs<float>& a, int nrhs, cudaStream_t s, float2* x,
                                      float2* r, float2* const* pbufs, const float2* q,
                                      cudaError_t (*zsweeps)(const PrecondArgs<float>&, int, cudaStream_t));
template <typename T> cudaError_t launch_sigma_large(const SigmaArgs<T>& a, int nrhs, cudaStream_t s);

// ---- launchers (defined in the .cu files) ----------------------------------

template <typename T> cudaError_t launch_stencil(const StencilArgs<T>& a, int nrhs, cudaStream_t s);
template <typename T> cudaError_t launch_sigma(const SigmaArgs<T>& a, int nrhs, cudaStream_t s);
// the self-energy as dense matrices (solver (b) of Sec. III; k_sigma_dense.cu)
int dense_row_tiles(int nf, int nxy);
cudaError_t build_sigma_dense(const double2* sigma, const double2* twx, const double2* twy, int nx,
                              int ny, int nf, int ne, double2* kscratch, float2* d32, double2* d64,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_sigma_dense(const SigmaArgs<T>& a, const typename Cplx<T>::type* D, int nrhs,
                               double2* part, int nslots_end, cudaStream_t s);
template <typename T> size_t sigma_smem_bytes(int nx, int ny, int threads);
template <typename T> cudaError_t launch_kb(const KbArgs<T>& a, int nrhs, cudaStream_t s);

// Krylov scalar and vector kernels
// pairs > 0: preconditioned Bi-CG on RHS pairs (i, i + pairs), i < pairs, the primary
// solving A x = b and its shadow A^T x~ = b~ (nrhs = 2 pairs).  rho = r~^T z and
// mu = p~^T q are the primary's partials (launch_pair_dot); both members share
// alpha, beta and their status (a pair stops, is replaced or breaks down together).
cudaError_t launch_beta(RhsState* st, const double2* rho_part, const double* rr_part, int nslots,
                        int slot_stride, int nrhs, int max_iter, double tol2, double delta2,
                        int mixed, cudaStream_t s, int pairs = 0);
cudaError_t launch_alpha(RhsState* st, const double2* mu_part, int nslots, int slot_stride,
                         int nrhs, cudaStream_t s, int pairs = 0);
// Bi-CG cross products: part[i][slot] = partials of a_{i+pairs}^T b_i for every pair i
// whose primary has a status in mask; a is the shadow's vector (or, with a_dir, a
// host array of the two direction buffers: the shadow's new direction
// a_dir[1 - pbuf]), b the primary's.  nslots equal chunks of the RHS.
template <typename T>
cudaError_t launch_pair_dot(const typename Cplx<T>::type* a, typename Cplx<T>::type* const* a_dir,
                            const typename Cplx<T>::type* b, const RhsState* st, int mask,
                            long long npts, int pairs, double2* part, int nslots, int slot_stride,
                            cudaStream_t s);
// dst[i] = src[i] * exp(i s kappa.r) for one vector (s = +1 or -1; phx[x] = exp(i kappa_x x h_x))
cudaError_t launch_gauge(double2* dst, const double2* src, const double2* phx, const double2* phy,
                         int sign, int nx, int ny, int nz, cudaStream_t s);
cudaError_t launch_restart_scalars(RhsState* st, const double2* rho_part, const double* rr_part,
                                   int nslots, int slot_stride, int nrhs, cudaStream_t s);
// x += alpha p, r -= alpha q with p = pbufs[pbuf] of each RHS
template <typename T>
cudaError_t launch_axpy_update(typename Cplx<T>::type* x, typename Cplx<T>::type* r,
                               typename Cplx<T>::type* const* pbufs,
                               const typename Cplx<T>::type* q, const RhsState* st, int mask,
                               long long npts, int nrhs, cudaStream_t s);
// The implicit operator form (free-propagator preconditioner M, A = M^{-1} - V - V_NL,
// z = M r): p = z + beta p_old into pbufs[1 - pbuf], q = (r - V z) + beta q in place, and
// the p^T q partials in slots [0, nz), one per plane (V_NL z is added by launch_kb with zsrc)
// With kb.nproj > 0 the pass also applies q -= V_NL z at the union points of each plane
// from the projections kb.sp that launch_kb_proj wrote before it.
template <typename T>
cudaError_t launch_pq_update(const typename Cplx<T>::type* z, const typename Cplx<T>::type* r,
                             typename Cplx<T>::type* const* pbufs, typename Cplx<T>::type* q,
                             const T* V, const RhsState* st, int mask, int nx, int ny, int nz,
                             int nrhs, double2* mu_part, int slot_stride, const KbArgs<T>& kb,
                             cudaStream_t s);
// the projections kb.sp[rhs][p] = E_p dvol <p|x> alone (x = kb.zsrc, or the operand of launch_kb)
template <typename T> cudaError_t launch_kb_proj(const KbArgs<T>& a, int nrhs, cudaStream_t s);
// x64 += x32; x32 = 0 (mixed-precision fold before the FP64 residual)
cudaError_t launch_fold(double2* x64, float2* x32, const RhsState* st, int mask, long long npts,
                        int nrhs, cudaStream_t s);
// r = b - y (y may be null) in FP64; writes r64 (may be null) and rT (element type T);
// rr partials per block.  yend (may be null): the end-plane terms -(Sigma x) kept apart
// by the self-energy (SigmaArgs::yend layout), added to y on those planes first.
template <typename T>
cudaError_t launch_residual(const double2* y, double2* r64, typename Cplx<T>::type* rT,
                            const RhsDesc* desc, const double2* phx, const double2* phy,
                            int nx, int ny, int nz, int nf, const RhsState* st, int mask,
                            double* rr_part, int slot_stride, int nrhs, cudaStream_t s,
                            int* nslots_out, const double2* yend = nullptr);
cudaError_t launch_set_status(RhsState* st, int nrhs, int from, int to, cudaStream_t s);
cudaError_t launch_status_cond(cudaGraphConditionalHandle cond, const RhsState* st, int nrhs,
                               int mask, cudaStream_t s);
cudaError_t launch_batch_cond(cudaGraphConditionalHandle cond, const RhsState* st, int nrhs,
                              int* counter, int max_chunks, cudaStream_t s);
cudaError_t launch_check(RhsState* st, const double* rr_part, int nslots, int slot_stride,
                         int nrhs, double tol2, int init, cudaStream_t s, int pairs = 0);
cudaError_t launch_projection(const double2* psi, const RhsDesc* desc, const int* open_ptr,
                              const int2* open_bins, const double2* phx, const double2* phy,
                              int nx, int ny, int nz, int nf, int max_open, double2* out,
                              int nrhs, cudaStream_t s);
// g(r) = 2 Re sum_o (sum_j L[o][j] Y_j(r)) (sum_k U[o][k] X_k(r))
cudaError_t launch_gradient(const double2* X, int nX, const double2* Y, int nY, const double2* U,
                            const double2* L, int n, long long npts, double* g, cudaStream_t s);
// dst = c1 * x1 + c2 * x2 (x2 may be null)
cudaError_t launch_combine(double2* dst, const double2* x1, double2 c1, const double2* x2,
                           double2 c2, long long npts, cudaStream_t s);

}  // namespace iobm

namespace iobm {
int stencil_slots(int nx, int ny, int nz, int zchunk, int nf);
}  // namespace iobm
