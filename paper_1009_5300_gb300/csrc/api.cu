// C ABI of the IOBM solver: handle management, the batched COCG driver
// (plain FP64 and mixed FP32/FP64 with FP64 residual replacement), channel
// projection, conductance and the adjoint gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <complex>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/iobm.h"
#include "iobm_internal.cuh"
#include "setup.h"

namespace iobm {
cudaError_t sigma_prepare();
}

using namespace iobm;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t n) {
        if (n <= bytes && p) return cudaSuccess;
        release();
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) bytes = n;
        return e;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

template <typename T>
cudaError_t upload(DevBuf& b, const std::vector<T>& v, cudaStream_t s) {
    cudaError_t e = b.ensure(sizeof(T) * std::max<size_t>(v.size(), 1));
    if (e != cudaSuccess) return e;
    if (v.empty()) return cudaSuccess;
    return cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s);
}

constexpr int kZChunkDefault = 32;   // z-planes per stencil CTA unless the autotuner picks another
constexpr int kZChunkMin = 16;       // smallest candidate: sizes the per-CTA partial-sum slots
// FP64 residual replacements run after every kReplaceEvery-th captured iteration
// (RHS that became PENDING wait at most kReplaceEvery - 1 iterations)
constexpr int kReplaceEvery = 2;
// z-segments (lanes) per mode of the double-float sweeps
constexpr int kZfSegments = 8;

}  // namespace

struct iobm_handle {
    iobm_grid g{};
    int nf = 4;
    double rs = 0.0;
    iobm_options opt{};
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;      // private stream (capturable)
    cudaStream_t cond_stream = nullptr; // captures the bodies of conditional graph nodes
    cudaStream_t side_stream = nullptr; // the double-float z-sweeps beside the FP32 ones
    cudaStream_t cond_side = nullptr;   // the same inside conditional bodies (a capture of their own)
    cudaEvent_t ev_zfork = nullptr, ev_zjoin = nullptr;
    cudaEvent_t ev_sfork = nullptr, ev_sjoin = nullptr;   // FP64 self-energy beside the stencil
    bool in_cond_body = false;          // launches go into a conditional node's body graph
    bool graph_conditionals = true;     // IF nodes around the residual replacements
    cudaEvent_t ev_sync = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    std::string err;
    long long npts = 0;
    int nxy = 0;
    std::vector<double> w;              // FD weights

    // persistent device tables
    DevBuf V32, V64;
    DevBuf errflag;                     // int, set by a kernel whose bounded wait gave up
    DevBuf twx32, twy32, twx64, twy64, phx, phy;
    FftAxis ax{}, ay{};
    ProjTables pt;
    DevBuf pptr, pidx, pval32, pval64, pcoup, uidx, uptr, uproj, uval32, uval64;

    // per-solve tables (handle owned)
    DevBuf sig32, sig64, pc32, pc64, ediag, rhs_energy, descs, open_ptr, open_bins, proj_out;
    DevBuf apply_sig32, apply_sig64, apply_pc32, apply_pc64, apply_ediag;
    std::vector<ModeTables> energies;
    std::vector<double> memo_E;          // energies of the tables kept by the last RHS count
    std::vector<ModeTables> memo_tables;
    std::vector<RhsDesc> hdesc;          // internal (real-profile) RHS
    std::vector<int> hrhs_energy;        // per internal RHS
    struct User {                        // one incident channel: psi = x[ic] + sign i x[is]
        int energy, chan, side, ic, is, sign;
    };
    std::vector<User> users;
    int side = 0;
    int nrhs = 0;                        // internal RHS
    int max_open = 0;
    // lateral Bloch vector (Eq. 8); nonzero: the solve runs in the gauge
    // phi = exp(-i kappa.r) psi as preconditioned Bi-CG on (kappa, -kappa) pairs
    double kappa[2] = {0.0, 0.0};
    int pairs = 0;                       // Bi-CG pairs of the current solve (0: COCG)
    DevBuf rhs_sign;                     // [nrhs] +1 / -1: the operator of each RHS is at s kappa
    DevBuf apply_sign;                   // [nrhs] +1 for iobm_apply
    DevBuf gph32, gph64;                 // [nxy] exp(i kappa.r_l) for the KB projectors
    DevBuf gpx, gpy;                     // [nx], [ny] exp(i kappa_x x h_x), exp(i kappa_y y h_y)
    DevBuf esc_rhs_sign;                 // the FP64 continuation's signs
    DevBuf zflag, zf_bins, zf_pc;        // FP64 z-sweep modes of the solve's energy slots
    int zf_k = 0;
    DevBuf zf_tab, zf_scr;               // their segment responses and scratch
    int zf_S = 1, zf_L = 0, zf_Lt = 0;
    long long wait_cycles = 0;           // bounded-wait limit of the bulk-copy kernels (0: default)
    int wait_inject = 0;                 // 1: their CTAs also wait on a barrier no copy completes
    int zchunk = kZChunkDefault;         // stencil z-planes per CTA (autotuned)
    int stencil_variant = 0;             // StencilArgs::variant (autotuned)
    DevBuf batch_ctr;                    // chunk counter of this junction in a batched solve
    DevBuf sig_scratch;                  // large-plane self-energy spectra
    DevBuf sig_end;                      // FP64 end-plane self-energy terms of the residual
    DevBuf kb_scratch;                  // KB projections [rhs][projector]
    DevBuf uplane;                      // [nz+1] first union-of-supports entry of each plane
    DevBuf esc_ws, esc_descs, esc_rhs_energy;   // FP64 continuation of stalled mixed RHS
    cudaGraphExec_t chunk_exec = nullptr;        // the last solve's chunk graph, updated in place
    void* pin = nullptr;                         // pinned staging buffer for table uploads
    size_t pin_bytes = 0;
    bool pc64_valid = false;                     // FP64 preconditioner tables of this solve uploaded
    // IOBM_SIGMA_DENSE: the dense self-energy matrices of the solve's energies and of
    // single applications, the FP64 lateral kernels they are filled from, tile partials
    DevBuf dense32, dense64, apply_dense32, apply_dense64, dense_k, dense_part;

    // workspace
    void* ws = nullptr;
    size_t ws_bytes = 0;
    DevBuf ws_owned;
    int ws_nrhs = 0;
    int ws_prec = -1;

    // layout of the current workspace
    int slot_stride = 0;
    int ns_stencil = 0;
    RhsState* st = nullptr;
    double2* mu_part = nullptr;
    double2* rho_part = nullptr;
    double* rr_part = nullptr;
    void* vx = nullptr;        // iterate (FP32 in mixed, FP64 in plain)
    void* vr = nullptr;
    void* vp[2] = {nullptr, nullptr};
    void* vq = nullptr;
    void* vz = nullptr;
    double2* x64 = nullptr;    // FP64 solution (mixed: separate; plain: == vx)
    double2* y64 = nullptr;
    bool solved = false;
    std::vector<RhsState> hstate;

    // stats
    double last_ms = 0.0;
    long long last_launches = 0;
    long long last_iters = 0;
    // optional in-graph CUDA-event timing of the fused stencil launches
    int profile = 0;
    std::vector<cudaEvent_t> kev;
    double prof_ms = 0.0;
    long long prof_launches = 0;
};

namespace {

int fail(iobm_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

int cuda_fail(iobm_handle* h, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, IOBM_E_CUDA, m);
}

#define CK(call)                                            \
    do {                                                    \
        cudaError_t _e = (call);                            \
        if (_e != cudaSuccess) return cuda_fail(h, _e, #call); \
    } while (0)

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

bool bloch(const iobm_handle* h) { return h->kappa[0] != 0.0 || h->kappa[1] != 0.0; }

// Internal (real-profile) RHS are solved to tol / sqrt(2): an incident channel
// psi = x_c +- i x_s then has ||b - A psi|| <= ||r_c|| + ||r_s|| <= tol ||b||
// because ||b||^2 = ||b_c||^2 + ||b_s||^2 (cos and sin profiles are orthogonal).
// At a lateral Bloch vector every channel is one internal RHS, solved to tol.
double internal_tol2(const iobm_handle* h) {
    return (bloch(h) ? 1.0 : 0.5) * h->opt.tol * h->opt.tol;
}

// per-RHS iteration limit of the current solve (the FP32 phase of a mixed solve
// stops at max_iter_mixed; the FP64 continuation gets max_iter)
int iter_cap(const iobm_handle* h) {
    return h->opt.precision == IOBM_MIXED ? std::min(h->opt.max_iter, h->opt.max_iter_mixed)
                                          : h->opt.max_iter;
}

// preconditioner applied through lateral plane FFTs (free propagator or Eq. 10)
bool fourier_precond(const iobm_handle* h) {
    return h->opt.use_precond == IOBM_PRECOND_FOURIER || h->opt.use_precond == IOBM_PRECOND_EQ10_FOURIER;
}

// q = A p through the free-propagator identity A z = r - V z - V_NL z (no stencil)
bool implicit_operator(const iobm_handle* h) {
    return h->opt.op_form == IOBM_OP_AUTO && h->opt.use_precond == IOBM_PRECOND_FOURIER;
}

bool large_plane(const iobm_handle* h) { return h->nxy > kSmemPlaneLimit; }

// partial slots per plane written by a plane transform (one per row block for
// the two-pass transforms of large planes)
int plane_slots(const iobm_handle* h) { return large_plane(h) ? large_row_blocks(h->g.ny) : 1; }

// mu partial slots of the self-energy
int sigma_slots(const iobm_handle* h) { return 2 * h->nf * plane_slots(h); }

bool dense_sigma(const iobm_handle* h) { return h->opt.sigma_form == IOBM_SIGMA_DENSE; }

// largest total of dense self-energy matrices (both precisions) a handle builds
constexpr double kDenseSigmaMaxBytes = 64.0 * (1ull << 30);

// The dense matrices (FP32 and FP64) of ne energies from their FP64 per-mode tables.
int build_dense_sigma(iobm_handle* h, const void* sig64, int ne, DevBuf& d32, DevBuf& d64) {
    const double M = (double)h->nf * h->nxy;
    const double bytes = (double)ne * M * M * (sizeof(float2) + sizeof(double2));
    if (bytes > kDenseSigmaMaxBytes)
        return fail(h, IOBM_E_UNSUPPORTED, "dense self-energy matrices above 64 GB");
    const size_t mm = (size_t)M * (size_t)M * (size_t)ne;
    CK(h->dense_k.ensure(sizeof(double2) * (size_t)ne * h->nf * h->nf * h->nxy));
    CK(d32.ensure(sizeof(float2) * mm));
    CK(d64.ensure(sizeof(double2) * mm));
    CK(build_sigma_dense((const double2*)sig64, h->twx64.as<double2>(), h->twy64.as<double2>(), h->g.nx,
                         h->g.ny, h->nf, ne, h->dense_k.as<double2>(), d32.as<float2>(),
                         d64.as<double2>(), h->stream));
    return IOBM_OK;
}

// y_end -= Sigma~ x_end: through the lateral FFT, or (IOBM_SIGMA_DENSE) by the dense
// matrices that belong to the per-mode tables `sig`
template <typename T>
int apply_sigma(iobm_handle* h, const SigmaArgs<T>& s, const void* sig, int nrhs) {
    if (!dense_sigma(h)) {
        CK(launch_sigma<T>(s, nrhs, h->stream));
        return IOBM_OK;
    }
    const bool f32 = std::is_same<T, float>::value;
    const DevBuf* D = nullptr;
    if (sig == h->sig32.p || sig == h->sig64.p) D = f32 ? &h->dense32 : &h->dense64;
    else if (sig == h->apply_sig32.p || sig == h->apply_sig64.p) D = f32 ? &h->apply_dense32 : &h->apply_dense64;
    if (!D || !D->p) return fail(h, IOBM_E_UNSUPPORTED, "dense self-energy matrices not built");
    if (s.dot_part && h->dense_part.bytes < sizeof(double2) * (size_t)nrhs * 2 *
                                                   dense_row_tiles(h->nf, h->nxy))
        return fail(h, IOBM_E_ARG, "dense self-energy partials not allocated for this RHS count");
    CK(launch_sigma_dense<T>(s, (const typename Cplx<T>::type*)D->p, nrhs, h->dense_part.as<double2>(),
                             h->nf * plane_slots(h), h->stream));
    return IOBM_OK;
}

int slots_for(const iobm_handle* h) {
    const int ns_op = stencil_slots(h->g.nx, h->g.ny, h->g.nz, kZChunkMin, h->nf);
    const int ns_pc = stencil_slots(h->g.nx, h->g.ny, h->g.nz, kZChunkMin, 1);
    const int kb = h->pt.nproj > 0 ? kb_slots((int)h->pt.uidx.size()) : 0;
    return std::max(std::max(ns_op + sigma_slots(h) + kb, 64),
                    std::max(std::max(h->g.nz * plane_slots(h), ns_pc), h->g.nz + kb));
}

// number of rho / |r|^2 partial slots the preconditioner pass writes
int rho_slots(const iobm_handle* h) {
    return fourier_precond(h)
               ? h->g.nz * plane_slots(h)
               : stencil_slots(h->g.nx, h->g.ny, h->g.nz, h->zchunk, 1);
}

// scratch of the large-plane self-energy (compact end-plane spectra, in and out)
cudaError_t ensure_sigma_scratch(iobm_handle* h, int nrhs) {
    if (h->pt.nproj > 0) {   // KB projections per (RHS, projector)
        const cudaError_t e = h->kb_scratch.ensure((size_t)std::max(nrhs, 1) * h->pt.nproj * sizeof(double2));
        if (e != cudaSuccess) return e;
    }
    if (dense_sigma(h)) {   // tile partials of the dense self-energy (per RHS, end, row tile)
        const cudaError_t e = h->dense_part.ensure(sizeof(double2) * (size_t)std::max(nrhs, 1) * 2 *
                                                   dense_row_tiles(h->nf, h->nxy));
        if (e != cudaSuccess) return e;
    }
    if (!large_plane(h)) {
        if (dense_sigma(h)) return cudaSuccess;
        // -(Sigma x) of the FP64 residual per (RHS, end, depth), formed beside the stencil
        return h->sig_end.ensure((size_t)std::max(nrhs, 1) * 2 * h->nf * h->nxy * sizeof(double2));
    }
    return h->sig_scratch.ensure(2 * (size_t)std::max(nrhs, 1) * 2 * h->nf * h->nxy * sizeof(double2));
}

size_t workspace_bytes(const iobm_handle* h, int nrhs, int prec) {
    const size_t n = (size_t)nrhs * h->npts;
    const int S = slots_for(h);
    size_t b = 0;
    b += align256(sizeof(RhsState) * nrhs);
    b += 2 * align256(sizeof(double2) * nrhs * S);
    b += align256(sizeof(double) * nrhs * S);
    const size_t ce = (prec == IOBM_MIXED) ? sizeof(float2) : sizeof(double2);
    b += 6 * align256(ce * n);                      // x r p0 p1 q z
    b += align256(sizeof(double2) * n);             // y64
    if (prec == IOBM_MIXED) b += align256(sizeof(double2) * n);   // x64
    return b;
}

int bind_workspace(iobm_handle* h, int nrhs) {
    const int prec = h->opt.precision;
    const size_t need = workspace_bytes(h, nrhs, prec);
    unsigned char* base = nullptr;
    if (h->ws && h->ws_bytes >= need) {
        base = reinterpret_cast<unsigned char*>(h->ws);
    } else {
        if (h->ws)
            return fail(h, IOBM_E_ARG, "attached workspace is smaller than iobm_workspace_size");
        cudaError_t e = h->ws_owned.ensure(need);
        if (e != cudaSuccess) return cuda_fail(h, e, "workspace allocation");
        base = h->ws_owned.as<unsigned char>();
    }
    const size_t n = (size_t)nrhs * h->npts;
    const int S = slots_for(h);
    h->slot_stride = S;
    h->ns_stencil = stencil_slots(h->g.nx, h->g.ny, h->g.nz, h->zchunk, h->nf);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void* p = base + off;
        off += align256(bytes);
        return p;
    };
    h->st = (RhsState*)take(sizeof(RhsState) * nrhs);
    h->mu_part = (double2*)take(sizeof(double2) * nrhs * S);
    h->rho_part = (double2*)take(sizeof(double2) * nrhs * S);
    h->rr_part = (double*)take(sizeof(double) * nrhs * S);
    const size_t ce = (prec == IOBM_MIXED) ? sizeof(float2) : sizeof(double2);
    h->vx = take(ce * n);
    h->vr = take(ce * n);
    h->vp[0] = take(ce * n);
    h->vp[1] = take(ce * n);
    h->vq = take(ce * n);
    h->vz = take(ce * n);
    h->y64 = (double2*)take(sizeof(double2) * n);
    h->x64 = (prec == IOBM_MIXED) ? (double2*)take(sizeof(double2) * n) : (double2*)h->vx;
    h->ws_nrhs = nrhs;
    h->ws_prec = prec;
    const cudaError_t e = ensure_sigma_scratch(h, nrhs);
    if (e != cudaSuccess) return cuda_fail(h, e, "self-energy scratch");
    return IOBM_OK;
}

// ---- argument blocks ---------------------------------------------------------

template <typename T>
StencilArgs<T> op_args(const iobm_handle* h) {
    StencilArgs<T> a{};
    a.nx = h->g.nx;
    a.ny = h->g.ny;
    a.nz = h->g.nz;
    a.nf = h->nf;
    const double ihx = 1.0 / (h->g.hx * h->g.hx), ihy = 1.0 / (h->g.hy * h->g.hy),
                 ihz = 1.0 / (h->g.hz * h->g.hz);
    auto pair = [](double c) {   // c as an FP32 pair hi + lo
        const float hi = (float)c;
        return make_float2(hi, (float)(c - (double)hi));
    };
    for (int n = 1; n <= h->nf; ++n) {
        a.cx[n] = (T)(0.5 * h->w[n] * ihx);
        a.cy[n] = (T)(0.5 * h->w[n] * ihy);
        a.cz[n] = (T)(0.5 * h->w[n] * ihz);
        a.dfx[n] = pair(0.5 * h->w[n] * ihx);
        a.dfy[n] = pair(0.5 * h->w[n] * ihy);
        a.dfz[n] = pair(0.5 * h->w[n] * ihz);
    }
    a.iso = 1;
    for (int n = 1; n <= h->nf; ++n) a.iso &= (a.cx[n] == a.cy[n] && a.cy[n] == a.cz[n]) ? 1 : 0;
    // difference form: the centre weight plus 2 sum_n c_n vanishes for the FD Laplacian
    a.c0 = (T)0;
    a.vsign = (T)(-1);
    a.V = std::is_same<T, float>::value ? (const T*)h->V32.p : (const T*)h->V64.p;
    a.npts = h->npts;
    a.zchunk = h->zchunk;
    a.variant = h->stencil_variant;
    a.mask = M_ALL;
    a.err = h->errflag.as<int>();
    a.wait_cycles = h->wait_cycles;
    a.wait_inject = h->wait_inject;
    if (std::is_same<T, double>::value && bloch(h)) {
        // lateral taps at the Bloch vector (FP64 kernels; per RHS the sign of kappa)
        a.rhs_sign = h->rhs_sign.as<int>();
        for (int n = 1; n <= h->nf; ++n) {
            const double tx = n * h->kappa[0] * h->g.hx, ty = n * h->kappa[1] * h->g.hy;
            const double cx = 0.5 * h->w[n] * ihx, cy = 0.5 * h->w[n] * ihy;
            a.bxc[n] = (T)(cx * std::cos(tx));
            a.bxs[n] = (T)(cx * std::sin(tx));
            a.byc[n] = (T)(cy * std::cos(ty));
            a.bys[n] = (T)(cy * std::sin(ty));
        }
    }
    return a;
}

template <typename T>
StencilArgs<T> precond_args(const iobm_handle* h) {
    StencilArgs<T> a{};
    a.nx = h->g.nx;
    a.ny = h->g.ny;
    a.nz = h->g.nz;
    a.nf = 1;
    const double c1 = h->opt.use_precond == IOBM_PRECOND_EQ10 ? std::exp(-h->opt.alpha) : 0.0;
    a.cx[1] = a.cy[1] = a.cz[1] = (T)c1;
    a.iso = 1;
    a.c0 = (T)(1.0 + 6.0 * c1);   // difference form: C_0 + 2 (3 C_1)
    a.vsign = (T)0;
    a.V = nullptr;
    a.npts = h->npts;
    a.zchunk = h->zchunk;
    a.variant = h->stencil_variant;
    a.mask = M_ALL;
    a.err = h->errflag.as<int>();
    a.wait_cycles = h->wait_cycles;
    a.wait_inject = h->wait_inject;
    return a;
}

template <typename T>
PrecondArgs<T> fourier_args(const iobm_handle* h, const void* pc) {
    PrecondArgs<T> a{};
    a.nx = h->g.nx;
    a.ny = h->g.ny;
    a.nz = h->g.nz;
    a.nf = h->nf;
    a.ax = h->ax;
    a.ay = h->ay;
    a.pc = (const typename Cplx<T>::type*)pc;
    if (std::is_same<T, float>::value) {
        a.twx = (const typename Cplx<T>::type*)h->twx32.p;
        a.twy = (const typename Cplx<T>::type*)h->twy32.p;
    } else {
        a.twx = (const typename Cplx<T>::type*)h->twx64.p;
        a.twy = (const typename Cplx<T>::type*)h->twy64.p;
    }
    a.npts = h->npts;
    a.mask = M_ALL;
    a.eq10 = (h->opt.use_precond == IOBM_PRECOND_EQ10_FOURIER) ? 1 : 0;
    a.c1 = std::exp(-h->opt.alpha);
    return a;
}

// the solve's FP64 z-sweep modes (FP32 iterations only; the tables follow the
// solve's energy slots, so single applications do not use them)
template <typename T>
void set_fp64_modes(const iobm_handle* h, PrecondArgs<T>& f) {
    if (!std::is_same<T, float>::value || h->zf_k <= 0) return;
    f.zflag = h->zflag.as<unsigned char>();
    f.zf_bins = h->zf_bins.as<int>();
    f.zf_pc = h->zf_pc.as<double2>();
    f.zf_k = h->zf_k;
    f.zf_tab = h->zf_tab.as<float4>();
    f.zf_scr = h->zf_scr.as<float4>();
    f.zf_S = h->zf_S;
    f.zf_L = h->zf_L;
    f.zf_Lt = h->zf_Lt;
    // the side stream joins the capture of the main graph when it forks there, so the
    // body of a conditional node (a capture of its own) forks to a side stream of its own
    f.zf_side = h->in_cond_body ? h->cond_side : h->side_stream;
    f.zf_fork = h->ev_zfork;
    f.zf_join = h->ev_zjoin;
}

template <typename T>
SigmaArgs<T> sigma_args(const iobm_handle* h, const void* sig) {
    SigmaArgs<T> a{};
    a.scratch = (typename Cplx<T>::type*)h->sig_scratch.p;
    a.nx = h->g.nx;
    a.ny = h->g.ny;
    a.nz = h->g.nz;
    a.nf = h->nf;
    a.ax = h->ax;
    a.ay = h->ay;
    a.sigma = (const typename Cplx<T>::type*)sig;
    if (std::is_same<T, float>::value) {
        a.twx = (const typename Cplx<T>::type*)h->twx32.p;
        a.twy = (const typename Cplx<T>::type*)h->twy32.p;
    } else {
        a.twx = (const typename Cplx<T>::type*)h->twx64.p;
        a.twy = (const typename Cplx<T>::type*)h->twy64.p;
    }
    a.npts = h->npts;
    a.mask = M_ALL;
    return a;
}

template <typename T>
KbArgs<T> kb_args(const iobm_handle* h) {
    KbArgs<T> a{};
    a.nproj = h->pt.nproj;
    a.pptr = h->pptr.as<int>();
    a.pidx = h->pidx.as<int>();
    a.pval = std::is_same<T, float>::value ? (const T*)h->pval32.p : (const T*)h->pval64.p;
    a.coupling = h->pcoup.as<double>();
    a.dvol = h->g.hx * h->g.hy * h->g.hz;
    a.nunion = (int)h->pt.uidx.size();
    a.uidx = h->uidx.as<int>();
    a.uptr = h->uptr.as<int>();
    a.uproj = h->uproj.as<int>();
    a.uval = std::is_same<T, float>::value ? (const T*)h->uval32.p : (const T*)h->uval64.p;
    a.npts = h->npts;
    a.mask = M_ALL;
    a.sp = (typename Cplx<T>::type*)h->kb_scratch.p;
    a.uplane = h->uplane.as<int>();
    a.nxy = h->nxy;
    if (bloch(h)) {
        a.rhs_sign = h->rhs_sign.as<int>();
        a.gph = std::is_same<T, float>::value ? (const typename Cplx<T>::type*)h->gph32.p
                                              : (const typename Cplx<T>::type*)h->gph64.p;
    }
    return a;
}

// y = A x (FP64 or FP32) for the RHS selected by (state, mask); energies per RHS.
// no_sigma: leave out the end-plane self-energy (the caller forms it apart).
template <typename T>
int apply_operator(iobm_handle* h, const void* x, void* y, int nrhs, const void* sig,
                   const double* ediag, const int* rhs_energy, const RhsState* st, int mask,
                   long long& launches, bool df = false, const int* signs = nullptr,
                   bool no_sigma = false) {
    using C = typename Cplx<T>::type;
    StencilArgs<T> a = op_args<T>(h);
    // FP64 data, double-float stencil arithmetic (the double-float kernel has no
    // Bloch phases: at a lateral Bloch vector the FP64 stencil runs instead)
    if (df && !bloch(h)) a.variant = 2;
    if (signs && std::is_same<T, double>::value && bloch(h)) a.rhs_sign = signs;
    a.x = (const C*)x;
    a.y = (C*)y;
    a.ediag = ediag;
    a.rhs_energy = rhs_energy;
    a.state = st;
    a.mask = mask;
    CK(launch_stencil<T>(a, nrhs, h->stream));
    launches += 1;
    if (!no_sigma) {
        SigmaArgs<T> s = sigma_args<T>(h, sig);
        s.x = (const C*)x;
        s.y = (C*)y;
        s.rhs_energy = rhs_energy;
        s.state = st;
        s.mask = mask;
        const int rc = apply_sigma<T>(h, s, sig, nrhs);
        if (rc) return rc;
        launches += 1;
    }
    if (h->pt.nproj > 0) {
        KbArgs<T> k = kb_args<T>(h);
        k.x = (const C*)x;
        k.y = (C*)y;
        k.state = st;
        k.mask = mask;
        if (signs && bloch(h)) k.rhs_sign = signs;
        CK(launch_kb<T>(k, nrhs, h->stream));
        launches += 2;
    }
    return IOBM_OK;
}

// Bi-CG: rho = r~^T z of every pair (primary partials) once z = P r is formed for
// the RHS in mask; the own r^T z partials of the preconditioner pass are replaced.
template <typename T>
int pair_rho(iobm_handle* h, int nrhs, int mask, long long& launches) {
    using C = typename Cplx<T>::type;
    if (!h->pairs) return IOBM_OK;
    (void)nrhs;
    CK(launch_pair_dot<T>((const C*)h->vr, nullptr, (const C*)h->vz, h->st, mask, h->npts, h->pairs,
                          h->rho_part, rho_slots(h), h->slot_stride, h->stream));
    launches += 1;
    return IOBM_OK;
}

// z = P r with rho = r^T z and rr = |r|^2 partials, for RHS in mask.
template <typename T>
int apply_precond_dots(iobm_handle* h, int nrhs, int mask, long long& launches) {
    using C = typename Cplx<T>::type;
    if (fourier_precond(h)) {
        PrecondArgs<T> f = fourier_args<T>(h, std::is_same<T, float>::value ? h->pc32.p : h->pc64.p);
        set_fp64_modes<T>(h, f);
        f.r = (const C*)h->vr;
        f.spec = (C*)h->vz;
        f.z = (C*)h->vz;
        f.rhs_energy = h->rhs_energy.as<int>();
        f.state = h->st;
        f.mask = mask;
        f.dot_part = h->rho_part;
        f.nrm_part = h->rr_part;
        f.slot_stride = h->slot_stride;
        CK(launch_precond_fourier<T>(f, nrhs, h->stream));
        launches += 3;
        return pair_rho<T>(h, nrhs, mask, launches);
    }
    StencilArgs<T> a = precond_args<T>(h);
    a.x = (const C*)h->vr;
    a.y = (C*)h->vz;
    a.state = h->st;
    a.mask = mask;
    a.dot_mode = 1;
    a.dot_part = h->rho_part;
    a.nrm_part = h->rr_part;
    a.slot_stride = h->slot_stride;
    a.slot_base = 0;
    CK(launch_stencil<T>(a, nrhs, h->stream));
    launches += 1;
    return pair_rho<T>(h, nrhs, mask, launches);
}

// FP64 residual r = b - A x64 of the RHS in `mask` into r (working precision) and
// its |r|^2 partials (*nslots per RHS).  The stencil (double-float when mixed) and
// the KB term run on h->stream; the end-plane self-energy, which reads only x64,
// runs beside them on a side stream into its own buffer, and the residual kernel
// adds it to y on the end planes: the same FP64 sums as when it updates y in place.
template <typename T>
int fp64_residual(iobm_handle* h, int nrhs, int mask, bool mixed, long long& launches, int* nslots) {
    using C = typename Cplx<T>::type;
    const bool apart = h->sig_end.p && !large_plane(h) && !dense_sigma(h) && !bloch(h);
    cudaStream_t side = h->in_cond_body ? h->cond_side : h->side_stream;
    if (apart) {
        CK(cudaEventRecord(h->ev_sfork, h->stream));
        CK(cudaStreamWaitEvent(side, h->ev_sfork, 0));
        SigmaArgs<double> s = sigma_args<double>(h, h->sig64.p);
        s.x = h->x64;
        s.y = h->y64;
        s.yend = h->sig_end.as<double2>();
        s.rhs_energy = h->rhs_energy.as<int>();
        s.state = h->st;
        s.mask = mask;
        CK(launch_sigma<double>(s, nrhs, side));
        CK(cudaEventRecord(h->ev_sjoin, side));
        launches += 1;
    }
    const int rc = apply_operator<double>(h, h->x64, h->y64, nrhs, h->sig64.p, h->ediag.as<double>(),
                                          h->rhs_energy.as<int>(), h->st, mask, launches, mixed,
                                          nullptr, apart);
    if (apart) CK(cudaStreamWaitEvent(h->stream, h->ev_sjoin, 0));   // joined even after a failure
    if (rc) return rc;
    CK(launch_residual<T>(h->y64, nullptr, (C*)h->vr, h->descs.as<RhsDesc>(), h->phx.as<double2>(),
                          h->phy.as<double2>(), h->g.nx, h->g.ny, h->g.nz, h->nf, h->st, mask,
                          h->rr_part, h->slot_stride, nrhs, h->stream, nslots,
                          apart ? h->sig_end.as<double2>() : nullptr));
    launches += 1;
    return IOBM_OK;
}

// FP64 residual replacement for RHS in `mask` (PENDING): x64 (+)= x, r = b - A x64.
template <typename T>
int residual_replacement(iobm_handle* h, int nrhs, int mask, bool mixed, long long& launches) {
    if (mixed) {
        CK(launch_fold(h->x64, (float2*)h->vx, h->st, mask, h->npts, nrhs, h->stream));
        launches += 1;
    }
    int nslots = 0;
    const int rc = fp64_residual<T>(h, nrhs, mask, mixed, launches, &nslots);
    if (rc) return rc;
    CK(launch_check(h->st, h->rr_part, nslots, h->slot_stride, nrhs, internal_tol2(h), 0, h->stream,
                    h->pairs));
    launches += 1;
    // RESTART RHS get z = P r and the rho / |r|^2 partials of the replaced residual;
    // the next iteration returns them to ACTIVE and forms beta from these partials
    return apply_precond_dots<T>(h, nrhs, M_RESTART, launches);
}

// Runs body() (launches on h->stream).  While h->stream is being captured the
// launches go into the body of a conditional IF node that executes only when
// some RHS has a status in `mask` when the graph reaches it (decided on the
// device), so the masked launches of steps that concern no RHS cost nothing.
//
// Kernel profilers cannot see the kernel nodes of graphs that hold conditional
// nodes: with IOBM_GRAPH_CONDITIONALS=0 in the environment at handle creation
// the steps are captured as plain masked launches instead (the same kernels on
// the same RHS, plus the launches that find no RHS to work on).
template <typename Body>
int captured_if_any(iobm_handle* h, int nrhs, int mask, Body body) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(h->stream, &cs));
    if (cs != cudaStreamCaptureStatusActive || !h->graph_conditionals) return body();
    cudaGraph_t cg = nullptr;
    CK(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, cg, 0, cudaGraphCondAssignDefault));
    CK(launch_status_cond(cond, h->st, nrhs, mask, h->stream));
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &cg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &p));
    CK(cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1,
                                           cudaStreamSetCaptureDependencies));
    CK(cudaStreamBeginCaptureToGraph(h->cond_stream, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    cudaStream_t main = h->stream;
    h->stream = h->cond_stream;
    h->in_cond_body = true;
    const int rc = body();
    h->in_cond_body = false;
    h->stream = main;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cond_stream, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(h, e, "conditional body capture");
    return IOBM_OK;
}

// One COCG iteration for every ACTIVE RHS.  Each RHS keeps its current
// direction in one of two buffers (RhsState::pbuf), so RHS that pause for an
// FP64 residual replacement resume with their own direction.
template <typename T>
int cocg_iteration(iobm_handle* h, int nrhs, bool mixed, long long& launches, int slot,
                   bool replace_now) {
    using C = typename Cplx<T>::type;
    const double tol2 = internal_tol2(h);
    const double delta2 = h->opt.refine_delta * h->opt.refine_delta;
    const int ns = h->ns_stencil;
    // RHS whose residual was replaced in the previous iteration resume here
    CK(launch_restart_scalars(h->st, h->rho_part, h->rr_part, h->ns_stencil, h->slot_stride, nrhs,
                              h->stream));
    CK(launch_beta(h->st, h->rho_part, h->rr_part, rho_slots(h), h->slot_stride, nrhs,
                   iter_cap(h), tol2, delta2, mixed ? 1 : 0, h->stream, h->pairs));
    launches += 2;
    // event record nodes inside the captured graph (external records execute with the graph)
    const bool timed = h->profile && slot >= 0;
    cudaEvent_t* kev = timed ? &h->kev[2 * slot] : nullptr;
    C* pb[2] = {(C*)h->vp[0], (C*)h->vp[1]};
    int nslots_mu = 0;
    if (implicit_operator(h)) {
        // projections of z, then p = z + beta p_old, q = (r - V z) + beta q_old - V_NL z
        KbArgs<T> k = kb_args<T>(h);   // nproj = 0: no KB term
        if (h->pt.nproj > 0) {
            k.zsrc = (const C*)h->vz;
            k.state = h->st;
            k.mask = M_ACTIVE;
            CK(launch_kb_proj<T>(k, nrhs, h->stream));
            launches += 1;
        }
        if (timed && h->profile == 1)
            CK(cudaEventRecordWithFlags(kev[0], h->stream, cudaEventRecordExternal));
        CK(launch_pq_update<T>((const C*)h->vz, (const C*)h->vr, pb, (C*)h->vq,
                               std::is_same<T, float>::value ? (const T*)h->V32.p : (const T*)h->V64.p,
                               h->st, M_ACTIVE, h->g.nx, h->g.ny, h->g.nz, nrhs, h->mu_part,
                               h->slot_stride, k, h->stream));
        if (timed && h->profile == 1)
            CK(cudaEventRecordWithFlags(kev[1], h->stream, cudaEventRecordExternal));
        nslots_mu = h->g.nz;   // one p^T q partial per plane
        launches += 1;
        if (h->pairs) {   // Bi-CG: mu = p~^T q with the shadow's new direction
            CK(launch_pair_dot<T>(nullptr, pb, (const C*)h->vq, h->st, M_ACTIVE, h->npts, h->pairs,
                                  h->mu_part, nslots_mu, h->slot_stride, h->stream));
            launches += 1;
        }
    } else {
        const void* sig = std::is_same<T, float>::value ? h->sig32.p : h->sig64.p;
        StencilArgs<T> a = op_args<T>(h);
        a.x = (const C*)h->vz;
        a.pbufs[0] = (C*)h->vp[0];
        a.pbufs[1] = (C*)h->vp[1];
        a.y = (C*)h->vq;
        a.fused_p = 1;
        a.ediag = h->ediag.as<double>();
        a.rhs_energy = h->rhs_energy.as<int>();
        a.state = h->st;
        a.mask = M_ACTIVE;
        a.dot_mode = 1;
        a.dot_part = h->mu_part;
        a.nrm_part = nullptr;
        a.slot_stride = h->slot_stride;
        a.slot_base = 0;
        if (timed && h->profile == 1)
            CK(cudaEventRecordWithFlags(kev[0], h->stream, cudaEventRecordExternal));
        CK(launch_stencil<T>(a, nrhs, h->stream));
        if (timed && h->profile == 1)
            CK(cudaEventRecordWithFlags(kev[1], h->stream, cudaEventRecordExternal));
        SigmaArgs<T> s = sigma_args<T>(h, sig);
        s.pnew[0] = (const C*)h->vp[0];
        s.pnew[1] = (const C*)h->vp[1];
        s.y = (C*)h->vq;
        s.rhs_energy = h->rhs_energy.as<int>();
        s.state = h->st;
        s.mask = M_ACTIVE;
        s.dot_part = h->mu_part;
        s.slot_stride = h->slot_stride;
        s.slot_base = ns;
        {
            const int rc = apply_sigma<T>(h, s, sig, nrhs);
            if (rc) return rc;
        }
        nslots_mu = ns + sigma_slots(h);
        launches += 3;
        if (h->pt.nproj > 0) {
            KbArgs<T> k = kb_args<T>(h);
            k.pnew[0] = (const C*)h->vp[0];
            k.pnew[1] = (const C*)h->vp[1];
            k.y = (C*)h->vq;
            k.state = h->st;
            k.mask = M_ACTIVE;
            k.dot_part = h->mu_part;
            k.slot_stride = h->slot_stride;
            k.slot_base = nslots_mu;
            CK(launch_kb<T>(k, nrhs, h->stream));
            nslots_mu += kb_slots(k.nunion);
            launches += 2;
        }
    }
    CK(launch_alpha(h->st, h->mu_part, nslots_mu, h->slot_stride, nrhs, h->stream, h->pairs));
    launches += 1;
    bool fused = false;
    if (fourier_precond(h)) {
        // x += alpha p, r -= alpha q fused with the forward plane FFTs of the preconditioner
        PrecondArgs<T> f = fourier_args<T>(h, std::is_same<T, float>::value ? h->pc32.p : h->pc64.p);
        set_fp64_modes<T>(h, f);
        f.r = (const C*)h->vr;
        f.spec = (C*)h->vz;
        f.z = (C*)h->vz;
        f.rhs_energy = h->rhs_energy.as<int>();
        f.state = h->st;
        f.mask = M_ACTIVE;
        f.dot_part = h->rho_part;
        f.nrm_part = h->rr_part;
        f.slot_stride = h->slot_stride;
        const cudaError_t e = launch_update_precond_fourier<T>(
            f, nrhs, h->stream, (C*)h->vx, (C*)h->vr, pb, (const C*)h->vq, kev,
            timed ? h->profile - 1 : 0);
        if (e == cudaSuccess) {
            fused = true;
            launches += 3;
            const int rc = pair_rho<T>(h, nrhs, M_ACTIVE, launches);
            if (rc) return rc;
        } else if (e != cudaErrorNotSupported) {
            return cuda_fail(h, e, "launch_update_precond_fourier");
        }
    }
    if (!fused) {
        CK(launch_axpy_update<T>((C*)h->vx, (C*)h->vr, pb, (const C*)h->vq, h->st, M_ACTIVE,
                                 h->npts, nrhs, h->stream));
        launches += 1;
        int rc = apply_precond_dots<T>(h, nrhs, M_ACTIVE, launches);
        if (rc) return rc;
    }
    // FP64 residual replacement of the RHS that became PENDING since the last one
    // (masked launches), every kReplaceEvery-th iteration of the captured chunk
    if (replace_now) {
        launches += 1;   // the condition kernel
        return captured_if_any(h, nrhs, M_PENDING, [&]() {
            return residual_replacement<T>(h, nrhs, M_PENDING, mixed, launches);
        });
    }
    return IOBM_OK;
}

// Reads (and clears) the kernels' error flag after the stream has drained.
int check_err_flag(iobm_handle* h) {
    int v = 0;
    CK(cudaMemcpyAsync(&v, h->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (v == 0) return IOBM_OK;
    CK(cudaMemsetAsync(h->errflag.p, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return fail(h, IOBM_E_TIMEOUT,
                "a kernel's bounded wait on its staged copies gave up (its CTA drained its own "
                "copies and returned; the results of this call are invalid)");
}

// Solver start for every RHS: zero x and the directions, r = b, ||b||^2, z = P r.
template <typename T>
int solver_prologue(iobm_handle* h, int nrhs, long long& launches) {
    using C = typename Cplx<T>::type;
    const bool mixed = std::is_same<T, float>::value;
    const size_t ce = sizeof(C);
    const size_t n = (size_t)nrhs * h->npts;
    CK(cudaEventRecord(h->ev_t0, h->stream));
    CK(cudaMemsetAsync(h->vx, 0, ce * n, h->stream));
    CK(cudaMemsetAsync(h->vp[0], 0, ce * n, h->stream));
    CK(cudaMemsetAsync(h->vp[1], 0, ce * n, h->stream));
    if (mixed) CK(cudaMemsetAsync(h->x64, 0, sizeof(double2) * n, h->stream));
    int nslots = 0;
    CK(launch_residual<T>(nullptr, nullptr, (C*)h->vr, h->descs.as<RhsDesc>(), h->phx.as<double2>(),
                          h->phy.as<double2>(), h->g.nx, h->g.ny, h->g.nz, h->nf, nullptr, M_ALL,
                          h->rr_part, h->slot_stride, nrhs, h->stream, &nslots));
    CK(launch_check(h->st, h->rr_part, nslots, h->slot_stride, nrhs, 0.0, 1, h->stream));
    launches += 2;
    return apply_precond_dots<T>(h, nrhs, M_RESTART, launches);
}

// Solver start from the iterate already in x (FP64 solver only, where x64 is x):
// ||b||^2 from r = b, then an FP64 residual replacement gives r = b - A x and
// z = P r for every RHS that is not already converged.
int solver_prologue_warm(iobm_handle* h, int nrhs, long long& launches) {
    using C = double2;
    const size_t n = (size_t)nrhs * h->npts;
    CK(cudaEventRecord(h->ev_t0, h->stream));
    CK(cudaMemsetAsync(h->vp[0], 0, sizeof(C) * n, h->stream));
    CK(cudaMemsetAsync(h->vp[1], 0, sizeof(C) * n, h->stream));
    int nslots = 0;
    CK(launch_residual<double>(nullptr, nullptr, (C*)h->vr, h->descs.as<RhsDesc>(), h->phx.as<double2>(),
                               h->phy.as<double2>(), h->g.nx, h->g.ny, h->g.nz, h->nf, nullptr, M_ALL,
                               h->rr_part, h->slot_stride, nrhs, h->stream, &nslots));
    CK(launch_check(h->st, h->rr_part, nslots, h->slot_stride, nrhs, 0.0, 1, h->stream));
    CK(launch_set_status(h->st, nrhs, ST_RESTART, ST_PENDING, h->stream));
    launches += 3;
    return residual_replacement<double>(h, nrhs, M_PENDING, false, launches);
}

// COCG iterations per captured chunk (a multiple of the replacement period)
int chunk_length(const iobm_handle* h) {
    return ((std::max(1, h->opt.chunk) + kReplaceEvery - 1) / kReplaceEvery) * kReplaceEvery;
}

// Launch one chunk of iterations on h->stream (which is being captured);
// timed: record the stencil event pairs (plain graphs only).
template <typename T>
int launch_chunk(iobm_handle* h, int nrhs, bool timed, long long& per_chunk) {
    const bool mixed = std::is_same<T, float>::value;
    const int chunk = chunk_length(h);
    for (int it = 0; it < chunk; ++it) {
        // iteration index `it` places the event pair (profiling) and the replacement
        const int rc = cocg_iteration<T>(h, nrhs, mixed, per_chunk, timed ? it : -1,
                                         (it + 1) % kReplaceEvery == 0);
        if (rc) return rc;
    }
    return IOBM_OK;
}

// Solver end: fold the FP32 progress of RHS that stopped without converging,
// record their FP64 residual, read the per-RHS state back.
template <typename T>
int solver_epilogue(iobm_handle* h, int nrhs, long long& launches) {
    const bool mixed = std::is_same<T, float>::value;
    const int mask = (1 << ST_NOCONV) | (1 << ST_BREAKDOWN) | (1 << ST_ACTIVE) | (1 << ST_PENDING) |
                     (1 << ST_RESTART);
    if (mixed) {
        CK(launch_fold(h->x64, (float2*)h->vx, h->st, mask, h->npts, nrhs, h->stream));
    }
    int nslots = 0;
    const int rc = fp64_residual<T>(h, nrhs, mask, mixed, launches, &nslots);
    if (rc) return rc;
    CK(launch_check(h->st, h->rr_part, nslots, h->slot_stride, nrhs, 0.0, 2, h->stream));
    CK(cudaEventRecord(h->ev_t1, h->stream));
    h->hstate.resize(nrhs);
    CK(cudaMemcpyAsync(h->hstate.data(), h->st, sizeof(RhsState) * nrhs, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1));
    h->last_ms = ms;
    h->last_launches = launches;
    long long it = 0;
    for (const RhsState& S : h->hstate) it += S.iters;
    h->last_iters = it;
    return check_err_flag(h);
}

template <typename T>
int run_solver(iobm_handle* h, int nrhs, bool warm = false) {
    long long launches = 0;
    int rc = (warm && !std::is_same<T, float>::value) ? solver_prologue_warm(h, nrhs, launches)
                                                      : solver_prologue<T>(h, nrhs, launches);
    if (rc) return rc;

    // capture one chunk of iterations
    const int chunk = chunk_length(h);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long per_chunk = 0;
    if (h->profile) {
        while ((int)h->kev.size() < 2 * chunk) {
            cudaEvent_t ev;
            CK(cudaEventCreate(&ev));
            h->kev.push_back(ev);
        }
    }
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    rc = launch_chunk<T>(h, nrhs, h->profile, per_chunk);
    if (rc) {
        cudaStreamEndCapture(h->stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    CK(cudaStreamEndCapture(h->stream, &graph));
    // the chunk of the previous solve usually has the same shape: update its
    // executable graph in place (new kernel arguments) instead of instantiating anew
    if (h->chunk_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(h->chunk_exec, graph, &info) == cudaSuccess) {
            exec = h->chunk_exec;
        } else {
            cudaGetLastError();
            cudaGraphExecDestroy(h->chunk_exec);
        }
        h->chunk_exec = nullptr;
    }
    if (!exec) {
        const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_fail(h, e, "cudaGraphInstantiate");
        }
    }
    cudaGraphDestroy(graph);

    h->hstate.resize(nrhs);
    const int max_chunks = iter_cap(h) / chunk + 4;
    int chunks = 0;
    for (; chunks < max_chunks; ++chunks) {
        cudaError_t e = cudaGraphLaunch(exec, h->stream);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            return cuda_fail(h, e, "cudaGraphLaunch");
        }
        launches += per_chunk;
        e = cudaMemcpyAsync(h->hstate.data(), h->st, sizeof(RhsState) * nrhs, cudaMemcpyDeviceToHost,
                            h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            return cuda_fail(h, e, "state readback");
        }
        if (h->profile) {
            for (int it = 0; it < chunk; ++it) {
                float kms = 0.f;
                if (cudaEventElapsedTime(&kms, h->kev[2 * it], h->kev[2 * it + 1]) == cudaSuccess) {
                    h->prof_ms += kms;
                    h->prof_launches += 1;
                } else {
                    cudaGetLastError();   // do not leave the failed query as the last error
                }
            }
        }
        int live = 0;
        for (const RhsState& S : h->hstate)
            live += (S.status == ST_ACTIVE || S.status == ST_RESTART || S.status == ST_PENDING);
        if (!live) break;
    }
    h->chunk_exec = exec;   // kept for the next solve
    return solver_epilogue<T>(h, nrhs, launches);
}

// Build the per-energy tables and the internal RHS list for energies E[0..nE).
// kind 0: incident channels (channels/nch) from `side`; kind 1: all forward
// channels at one energy followed by the adjoint functionals of every channel.
// An incident channel exp(i G.r) is run as the real profiles cos(G.r) and
// sin(G.r) of its +-G pair (one profile for a self-conjugate G).
int upload_solve_tables(iobm_handle* h);
int prepare_rhs_bloch(iobm_handle* h, const double* E, int nE, const int* channels, int nch,
                      int side, int kind, bool upload_tables);

int prepare_rhs(iobm_handle* h, const double* E, int nE, const int* channels, int nch, int side,
                int kind, bool upload_tables = true) {
    if (bloch(h)) return prepare_rhs_bloch(h, E, nE, channels, nch, side, kind, upload_tables);
    h->pairs = 0;
    h->energies.clear();
    h->hdesc.clear();
    h->hrhs_energy.clear();
    h->users.clear();
    h->side = side;
    const int nf = h->nf;
    auto add_desc = [&](int e, const ModeTables& mt, int q, int side_, int profile,
                        const std::complex<double>* coef, double scale) {
        RhsDesc d{};
        d.energy = e;
        d.kx = mt.open_kx[q];
        d.ky = mt.open_ky[q];
        d.side = side_;
        d.profile = profile;
        for (int k = 0; k < nf; ++k) d.coef[k] = make_double2(scale * coef[k].real(), scale * coef[k].imag());
        h->hdesc.push_back(d);
        h->hrhs_energy.push_back(e);
        return (int)h->hdesc.size() - 1;
    };
    for (int e = 0; e < nE; ++e)
        if (!std::isfinite(E[e])) return fail(h, IOBM_E_ARG, "non-finite energy");
    std::vector<ModeTables> tables;
    const bool memo_hit = upload_tables && (int)h->memo_E.size() == nE &&
                          std::equal(h->memo_E.begin(), h->memo_E.end(), E);
    if (memo_hit) {
        tables = std::move(h->memo_tables);
    } else {
        std::string msg;
        // a count (no upload) builds the full tables too, for the solve that follows it
        const int rc = build_mode_tables_many(h->g.nx, h->g.ny, h->g.hx, h->g.hy, h->g.hz, nf, E, nE,
                                              true, tables, msg);
        if (rc) return fail(h, rc == 2 ? IOBM_E_THRESHOLD : IOBM_E_UNSUPPORTED, msg);
    }
    h->memo_E.clear();
    h->memo_tables.clear();
    for (int e = 0; e < nE; ++e) {
        ModeTables& mt = tables[e];
        std::vector<int> list;
        if (kind == 1 || !channels) {
            for (int c = 0; c < mt.nopen; ++c) list.push_back(c);
        } else {
            for (int c = 0; c < nch; ++c)
                if (channels[c] >= 0 && channels[c] < mt.nopen &&
                    std::find(list.begin(), list.end(), channels[c]) == list.end())
                    list.push_back(channels[c]);
        }
        // pairs {q, partner(q)} with q the smaller index
        std::vector<int> roots;
        for (int c : list) {
            const int q = std::min(c, mt.open_partner[c]);
            if (std::find(roots.begin(), roots.end(), q) == roots.end()) roots.push_back(q);
        }
        std::sort(roots.begin(), roots.end());
        const int fside = (kind == 1) ? 0 : side;
        std::vector<int> icos(mt.nopen, -1), isin(mt.nopen, -1);
        for (int q : roots) {
            const std::complex<double>* b = &mt.btilde[(size_t)q * nf];
            icos[q] = add_desc(e, mt, q, fside, PROF_COS, b, 1.0);
            if (mt.open_partner[q] != q) isin[q] = add_desc(e, mt, q, fside, PROF_SIN, b, 1.0);
        }
        std::sort(list.begin(), list.end());
        for (int c : list) {
            const int q = std::min(c, mt.open_partner[c]);
            iobm_handle::User u{};
            u.energy = e;
            u.chan = c;
            u.side = fside;
            u.ic = icos[q];
            u.is = isin[q];
            u.sign = (c == q) ? +1 : -1;
            h->users.push_back(u);
        }
        if (kind == 1) {
            // adjoint functionals w_o = mrow_o exp(-i G_o.r) / N_xy on the exit planes
            const double inv = 1.0 / h->nxy;
            for (int q : roots) {
                const std::complex<double>* m = &mt.mrow[(size_t)q * nf];
                add_desc(e, mt, q, 1 - fside, PROF_COS, m, inv);
                if (mt.open_partner[q] != q) add_desc(e, mt, q, 1 - fside, PROF_SIN, m, inv);
            }
        }
        h->energies.push_back(std::move(mt));
    }
    h->nrhs = (int)h->hdesc.size();
    if (!upload_tables) {
        // keep the tables for the solve that normally follows a count
        h->memo_E.assign(E, E + nE);
        h->memo_tables = std::move(h->energies);
        h->energies.clear();
        return IOBM_OK;
    }
    return upload_solve_tables(h);
}

// Device copies of the per-energy-slot tables, energies, RHS descriptors and
// open-channel lists of the RHS list just built (h->energies, h->hdesc, ...).
int upload_solve_tables(iobm_handle* h) {
    const int nE = (int)h->energies.size();
    // device tables, staged through pinned memory: Sigma~ in FP32 and FP64, the
    // free-propagator factors in FP32 (FP64 only for an FP64 solve; the FP64
    // continuation of a mixed solve uploads them when it needs them)
    size_t nsig = 0, npc = 0;
    for (const ModeTables& mt : h->energies) {
        nsig += mt.sigma.size();
        npc += mt.pc.size();
    }
    const bool pc64_now = h->opt.precision == IOBM_FP64;
    const size_t pin_need = nsig * (sizeof(double2) + sizeof(float2)) +
                            npc * (sizeof(float2) + (pc64_now ? sizeof(double2) : 0)) + 64;
    if (h->pin_bytes < pin_need) {
        if (h->pin) cudaFreeHost(h->pin);
        h->pin = nullptr;
        h->pin_bytes = 0;
        CK(cudaMallocHost(&h->pin, pin_need));
        h->pin_bytes = pin_need;
    }
    CK(cudaStreamSynchronize(h->stream));   // the previous uploads from the staging buffer are done
    double2* s64 = reinterpret_cast<double2*>(h->pin);
    float2* s32 = reinterpret_cast<float2*>(s64 + nsig);
    float2* p32 = s32 + nsig;
    double2* p64 = reinterpret_cast<double2*>(p32 + npc);
    {
        size_t is = 0, ip = 0;
        for (const ModeTables& mt : h->energies) {
            for (const auto& v : mt.sigma) {
                s64[is] = make_double2(v.real(), v.imag());
                s32[is] = make_float2((float)v.real(), (float)v.imag());
                ++is;
            }
            for (const auto& v : mt.pc) {
                p32[ip] = make_float2((float)v.real(), (float)v.imag());
                if (pc64_now) p64[ip] = make_double2(v.real(), v.imag());
                ++ip;
            }
        }
    }
    auto put = [&](DevBuf& b, const void* src, size_t bytes) -> cudaError_t {
        cudaError_t e = b.ensure(std::max<size_t>(bytes, 16));
        if (e == cudaSuccess && bytes)
            e = cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, h->stream);
        return e;
    };
    CK(put(h->sig64, s64, sizeof(double2) * nsig));
    CK(put(h->sig32, s32, sizeof(float2) * nsig));
    if (dense_sigma(h)) {
        const int rc = build_dense_sigma(h, h->sig64.p, (int)h->energies.size(), h->dense32, h->dense64);
        if (rc) return rc;
    }
    CK(put(h->pc32, p32, sizeof(float2) * npc));
    if (pc64_now) CK(put(h->pc64, p64, sizeof(double2) * npc));
    h->pc64_valid = pc64_now;
    std::vector<double> ed(nE);
    std::vector<int> optr(nE + 1, 0);
    std::vector<int2> obins;
    h->max_open = 0;
    for (int e = 0; e < nE; ++e) {
        ed[e] = h->energies[e].E;
        const ModeTables& mt = h->energies[e];
        optr[e + 1] = optr[e] + mt.nopen;
        h->max_open = std::max(h->max_open, mt.nopen);
        for (int c = 0; c < mt.nopen; ++c) obins.push_back(make_int2(mt.open_kx[c], mt.open_ky[c]));
    }
    CK(upload(h->ediag, ed, h->stream));
    CK(upload(h->rhs_energy, h->hrhs_energy, h->stream));
    CK(upload(h->descs, h->hdesc, h->stream));
    CK(upload(h->open_ptr, optr, h->stream));
    CK(upload(h->open_bins, obins, h->stream));
    if (h->pairs) {
        std::vector<int> sg(h->nrhs);
        for (int i = 0; i < h->nrhs; ++i) sg[i] = i < h->pairs ? 1 : -1;
        CK(upload(h->rhs_sign, sg, h->stream));
    }
    // per energy slot the fp64_modes lateral modes nearest their threshold (smallest
    // |E - eps_perp|, ties by bin): FP64 z-sweeps in the FP32 iterations
    const int want = h->opt.fp64_modes >= 0 ? h->opt.fp64_modes : std::max(16, h->nxy / 128);
    h->zf_k = (h->opt.precision == IOBM_MIXED && fourier_precond(h) &&
               h->opt.use_precond == IOBM_PRECOND_FOURIER)
                  ? std::min(want, h->nxy) : 0;
    if (h->zf_k > 0) {
        const int K = h->zf_k, nxy = h->nxy;
        std::vector<unsigned char> flag((size_t)nE * nxy, 0);
        std::vector<int> bins((size_t)nE * K);
        std::vector<double2> zpc((size_t)nE * K * kPcStrideDev);
        std::vector<int> order(nxy);
        for (int e = 0; e < nE; ++e) {
            const ModeTables& mt = h->energies[e];
            for (int b = 0; b < nxy; ++b) order[b] = b;
            std::partial_sort(order.begin(), order.begin() + K, order.end(), [&](int a, int b) {
                const double da = std::fabs(mt.E - mt.eperp_bin[a]), db = std::fabs(mt.E - mt.eperp_bin[b]);
                return da < db || (da == db && a < b);
            });
            for (int f = 0; f < K; ++f) {
                const int b = order[f];
                flag[(size_t)e * nxy + b] = 1;
                bins[(size_t)e * K + f] = b;
                for (int j = 0; j < kPcStrideDev; ++j) {
                    const std::complex<double> v = mt.pc[(size_t)b * kPcStride + j];
                    zpc[((size_t)e * K + f) * kPcStrideDev + j] = make_double2(v.real(), v.imag());
                }
            }
        }
        CK(upload(h->zflag, flag, h->stream));
        CK(upload(h->zf_bins, bins, h->stream));
        CK(upload(h->zf_pc, zpc, h->stream));
        // z-segments of the double-float sweeps: at most kZfSegments, each >= nf planes,
        // the last one absorbing the remainder (< L + nf planes)
        const int NF = h->nf, m = h->g.nz - NF;
        int S = std::max(1, std::min(kZfSegments, m / NF));
        int L = (m + S - 1) / S;
        while (S > 1 && m - (S - 1) * L < NF) --S;
        if (S > 1) L = std::max(L, NF);
        h->zf_S = S;
        h->zf_L = S > 1 ? L : m;
        h->zf_Lt = S > 1 ? L + NF : m;
        const int Lt = h->zf_Lt;
        // responses h_j (j < Lt) of h_j = sum_t c_t h_{j-t} to the history h_{-1-i} = 1:
        // forward c_t = -l_t, backward c_t = -u_t / u_0 (the factors of the sweeps)
        std::vector<float4> tab((size_t)nE * K * 2 * NF * Lt);
        auto split = [](std::complex<double> v) {
            const float hr = (float)v.real(), hi = (float)v.imag();
            return make_float4(hr, hi, (float)(v.real() - (double)hr), (float)(v.imag() - (double)hi));
        };
        std::vector<std::complex<double>> hv(Lt + NF);
        for (int e = 0; e < nE; ++e)
            for (int f = 0; f < K; ++f) {
                const double2* pc = &zpc[((size_t)e * K + f) * kPcStrideDev];
                std::complex<double> c[2][5];
                const std::complex<double> u0(pc[NF].x, pc[NF].y);
                for (int t = 1; t <= NF; ++t) {
                    c[0][t] = -std::complex<double>(pc[t - 1].x, pc[t - 1].y);
                    c[1][t] = -std::complex<double>(pc[NF + t].x, pc[NF + t].y) / u0;
                }
                for (int d = 0; d < 2; ++d)
                    for (int i = 0; i < NF; ++i) {
                        // hv[NF + j] = h_j; hv[NF - 1 - i'] = history h_{-1-i'}
                        std::fill(hv.begin(), hv.end(), std::complex<double>(0.0, 0.0));
                        hv[NF - 1 - i] = 1.0;
                        for (int j = 0; j < Lt; ++j) {
                            std::complex<double> acc(0.0, 0.0);
                            for (int t = 1; t <= NF; ++t) acc += c[d][t] * hv[NF + j - t];
                            hv[NF + j] = acc;
                            tab[((((size_t)e * K + f) * 2 + d) * NF + i) * Lt + j] = split(acc);
                        }
                    }
            }
        CK(upload(h->zf_tab, tab, h->stream));
        CK(h->zf_scr.ensure(sizeof(float4) * (size_t)std::max(h->nrhs, 1) * K * m));
    }
    return IOBM_OK;
}


// The RHS list at a lateral Bloch vector kappa (Eq. 8), solved in the gauge
// phi = exp(-i kappa.r) psi, where the operator A(kappa) has A(kappa)^T = A(-kappa):
// energy slots [0, nE) hold the tables at +kappa (modes G_nu + kappa), slots
// [nE, 2 nE) those at -kappa.  Every internal RHS is one incident channel (source
// exp(i G_nu.r) b~ in the gauge, no real-profile pairing) and RHS i + pairs is the
// Bi-CG shadow of RHS i: kind 0, the channel -nu of -kappa incident from the same
// side (time-reversed partner; its solution is the -kappa problem's wave); kind 1
// (gradient, one energy), the adjoint functional w_o of the same channel o, whose
// shadow solution is lambda_o = A(kappa)^{-T} w_o in the gauge of -kappa.
int prepare_rhs_bloch(iobm_handle* h, const double* E, int nE, const int* channels, int nch,
                      int side, int kind, bool upload_tables) {
    h->energies.clear();
    h->hdesc.clear();
    h->hrhs_energy.clear();
    h->users.clear();
    h->side = side;
    const int nf = h->nf;
    for (int e = 0; e < nE; ++e)
        if (!std::isfinite(E[e])) return fail(h, IOBM_E_ARG, "non-finite energy");
    std::vector<ModeTables> tables;
    const bool memo_hit = upload_tables && (int)h->memo_E.size() == nE &&
                          (int)h->memo_tables.size() == 2 * nE &&
                          std::equal(h->memo_E.begin(), h->memo_E.end(), E);
    if (memo_hit) {
        tables = std::move(h->memo_tables);
    } else {
        std::string msg;
        std::vector<ModeTables> minus;
        int rc = build_mode_tables_many(h->g.nx, h->g.ny, h->g.hx, h->g.hy, h->g.hz, nf, E, nE, true,
                                        tables, msg, h->kappa[0], h->kappa[1]);
        if (!rc)
            rc = build_mode_tables_many(h->g.nx, h->g.ny, h->g.hx, h->g.hy, h->g.hz, nf, E, nE, true,
                                        minus, msg, -h->kappa[0], -h->kappa[1]);
        if (rc) return fail(h, rc == 2 ? IOBM_E_THRESHOLD : IOBM_E_UNSUPPORTED, msg);
        for (ModeTables& mt : minus) tables.push_back(std::move(mt));
    }
    h->memo_E.clear();
    h->memo_tables.clear();
    auto add_desc = [&](int slot, int kx, int ky, int side_, const std::complex<double>* coef,
                        double scale) {
        RhsDesc d{};
        d.energy = slot;
        d.kx = kx;
        d.ky = ky;
        d.side = side_;
        d.profile = PROF_EXP_PLUS;
        for (int k = 0; k < nf; ++k) d.coef[k] = make_double2(scale * coef[k].real(), scale * coef[k].imag());
        h->hdesc.push_back(d);
        h->hrhs_energy.push_back(slot);
    };
    // index, in the open list of a -kappa slot, of the channel with lateral index -nu
    auto partner = [&](const ModeTables& mm, const ModeTables& mp, int c) {
        const int bx = (h->g.nx - mp.open_kx[c]) % h->g.nx, by = (h->g.ny - mp.open_ky[c]) % h->g.ny;
        for (int d = 0; d < mm.nopen; ++d)
            if (mm.open_kx[d] == bx && mm.open_ky[d] == by) return d;
        return -1;
    };
    struct Item { int e, c, cm; };
    std::vector<Item> items;
    for (int e = 0; e < nE; ++e) {
        const ModeTables& mp = tables[e];
        const ModeTables& mm = tables[nE + e];
        if (mm.nopen != mp.nopen)
            return fail(h, IOBM_E_UNSUPPORTED, "open channels of +kappa and -kappa differ");
        std::vector<int> list;
        if (kind == 1 || !channels) {
            for (int c = 0; c < mp.nopen; ++c) list.push_back(c);
        } else {
            for (int c = 0; c < nch; ++c)
                if (channels[c] >= 0 && channels[c] < mp.nopen &&
                    std::find(list.begin(), list.end(), channels[c]) == list.end())
                    list.push_back(channels[c]);
            std::sort(list.begin(), list.end());
        }
        for (int c : list) {
            const int cm = partner(mm, mp, c);
            if (cm < 0) return fail(h, IOBM_E_UNSUPPORTED, "open channel without a -nu partner at -kappa");
            items.push_back({e, c, cm});
        }
    }
    const int fside = (kind == 1) ? 0 : side;
    const int n = (int)items.size();
    h->pairs = n;
    for (int i = 0; i < n; ++i) {   // primaries: the channels at +kappa
        const ModeTables& mp = tables[items[i].e];
        const int c = items[i].c;
        add_desc(items[i].e, mp.open_kx[c], mp.open_ky[c], fside, &mp.btilde[(size_t)c * nf], 1.0);
        h->users.push_back({items[i].e, c, fside, i, -1, 1});
    }
    for (int i = 0; i < n; ++i) {   // shadows
        const ModeTables& mp = tables[items[i].e];
        const ModeTables& mm = tables[nE + items[i].e];
        if (kind == 1) {
            // w_o = mrow_o exp(-i (G_o + kappa).r) / N_xy on the exit planes; in the
            // gauge of -kappa this is exp(i G_{-nu}.r) mrow_o / N_xy
            const int c = items[i].c;
            add_desc(nE + items[i].e, (h->g.nx - mp.open_kx[c]) % h->g.nx,
                     (h->g.ny - mp.open_ky[c]) % h->g.ny, 1 - fside, &mp.mrow[(size_t)c * nf],
                     1.0 / h->nxy);
        } else {
            const int cm = items[i].cm;
            add_desc(nE + items[i].e, mm.open_kx[cm], mm.open_ky[cm], fside,
                     &mm.btilde[(size_t)cm * nf], 1.0);
            h->users.push_back({nE + items[i].e, cm, fside, n + i, -1, 1});
        }
    }
    h->energies = std::move(tables);
    h->nrhs = (int)h->hdesc.size();
    if (!upload_tables) {
        h->memo_E.assign(E, E + nE);
        h->memo_tables = std::move(h->energies);
        h->energies.clear();
        return IOBM_OK;
    }
    return upload_solve_tables(h);
}

// Precision escalation after a mixed solve: the RHS that stopped without
// converging (FP32 iteration limit or breakdown) are solved again with FP64
// COCG, starting from their FP64 iterate, in a separate FP64 workspace; their
// solutions, states and counts are merged back.  The handle's workspace
// bindings are swapped for the sub-solve and restored afterwards.
int escalate_fp64(iobm_handle* h) {
    std::vector<int> idx;
    for (int i = 0; i < h->nrhs; ++i) {
        const int st = h->hstate[i].status;
        if (st == ST_NOCONV || st == ST_BREAKDOWN) idx.push_back(i);
    }
    if (idx.empty()) return IOBM_OK;
    const int m = (int)idx.size();
    if (!h->pc64_valid) {   // FP64 free-propagator factors for the FP64 iterations
        std::vector<double2> p64;
        for (const ModeTables& mt : h->energies)
            for (const auto& v : mt.pc) p64.push_back(make_double2(v.real(), v.imag()));
        CK(upload(h->pc64, p64, h->stream));
        h->pc64_valid = true;
    }
    // Bi-CG pairs stop together, so the stalled set holds whole pairs: its primaries
    // (indices below pairs) come first, their shadows after in the same order
    const int sub_pairs = h->pairs ? m / 2 : 0;
    std::vector<RhsDesc> sd(m);
    std::vector<int> se(m), ss(m);
    for (int k = 0; k < m; ++k) {
        sd[k] = h->hdesc[idx[k]];
        se[k] = h->hrhs_energy[idx[k]];
        ss[k] = k < sub_pairs ? 1 : -1;
    }
    CK(upload(h->esc_descs, sd, h->stream));
    CK(upload(h->esc_rhs_energy, se, h->stream));
    if (h->pairs) CK(upload(h->esc_rhs_sign, ss, h->stream));
    const size_t need = workspace_bytes(h, m, IOBM_FP64);
    CK(h->esc_ws.ensure(need));

    struct Saved {
        void* ws; size_t ws_bytes; int ws_nrhs, ws_prec, slot_stride, ns_stencil, nrhs, precision;
        RhsState* st; double2 *mu_part, *rho_part; double* rr_part;
        void *vx, *vr, *vp0, *vp1, *vq, *vz; double2 *x64, *y64;
        double last_ms; long long last_launches, last_iters; int profile, pairs;
    } sv{h->ws, h->ws_bytes, h->ws_nrhs, h->ws_prec, h->slot_stride, h->ns_stencil, h->nrhs,
         h->opt.precision, h->st, h->mu_part, h->rho_part, h->rr_part, h->vx, h->vr, h->vp[0],
         h->vp[1], h->vq, h->vz, h->x64, h->y64, h->last_ms, h->last_launches, h->last_iters,
         h->profile, h->pairs};
    std::vector<RhsState> main_state = h->hstate;
    auto restore = [&]() {
        h->ws = sv.ws; h->ws_bytes = sv.ws_bytes; h->ws_nrhs = sv.ws_nrhs; h->ws_prec = sv.ws_prec;
        h->slot_stride = sv.slot_stride; h->ns_stencil = sv.ns_stencil; h->nrhs = sv.nrhs;
        h->opt.precision = sv.precision; h->st = sv.st; h->mu_part = sv.mu_part;
        h->rho_part = sv.rho_part; h->rr_part = sv.rr_part; h->vx = sv.vx; h->vr = sv.vr;
        h->vp[0] = sv.vp0; h->vp[1] = sv.vp1; h->vq = sv.vq; h->vz = sv.vz; h->x64 = sv.x64;
        h->y64 = sv.y64; h->profile = sv.profile; h->pairs = sv.pairs;
        std::swap(h->descs, h->esc_descs);
        std::swap(h->rhs_energy, h->esc_rhs_energy);
        if (sv.pairs) std::swap(h->rhs_sign, h->esc_rhs_sign);
    };
    std::swap(h->descs, h->esc_descs);
    std::swap(h->rhs_energy, h->esc_rhs_energy);
    if (h->pairs) std::swap(h->rhs_sign, h->esc_rhs_sign);
    h->pairs = sub_pairs;
    h->ws = h->esc_ws.p;
    h->ws_bytes = need;
    h->opt.precision = IOBM_FP64;
    h->nrhs = m;
    h->profile = 0;
    int rc = bind_workspace(h, m);
    // the FP64 iterate of every stalled RHS is the starting point
    for (int k = 0; !rc && k < m; ++k) {
        const cudaError_t e = cudaMemcpyAsync((double2*)h->vx + (size_t)k * h->npts,
                                              sv.x64 + (size_t)idx[k] * h->npts,
                                              sizeof(double2) * h->npts, cudaMemcpyDeviceToDevice,
                                              h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "escalation start");
    }
    if (!rc) rc = run_solver<double>(h, m, true);
    for (int k = 0; !rc && k < m; ++k) {
        const cudaError_t e = cudaMemcpyAsync(sv.x64 + (size_t)idx[k] * h->npts,
                                              (double2*)h->vx + (size_t)k * h->npts,
                                              sizeof(double2) * h->npts, cudaMemcpyDeviceToDevice,
                                              h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "escalation result");
    }
    const std::vector<RhsState> sub = h->hstate;
    const double sub_ms = h->last_ms;
    const long long sub_launches = h->last_launches, sub_iters = h->last_iters;
    restore();
    h->hstate = main_state;
    if (rc) return rc;
    for (int k = 0; k < m; ++k) {
        RhsState& S = h->hstate[idx[k]];
        const int iters = S.iters, reps = S.replacements;
        S = sub[k];
        S.iters += iters;
        S.replacements += reps;
    }
    CK(cudaMemcpyAsync(h->st, h->hstate.data(), sizeof(RhsState) * h->nrhs, cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->last_ms = sv.last_ms + sub_ms;
    h->last_launches = sv.last_launches + sub_launches;
    h->last_iters = sv.last_iters + sub_iters;
    return IOBM_OK;
}

// projection sums of the FP64 solutions (Eq. 19 on the end planes) after a solve
int launch_projections(iobm_handle* h) {
    const size_t pbytes = sizeof(double2) * (size_t)h->nrhs * std::max(h->max_open, 1) * 2 * kMaxNf;
    CK(h->proj_out.ensure(pbytes));
    CK(launch_projection(h->x64, h->descs.as<RhsDesc>(), h->open_ptr.as<int>(), h->open_bins.as<int2>(),
                         h->phx.as<double2>(), h->phy.as<double2>(), h->g.nx, h->g.ny, h->g.nz,
                         h->nf, h->max_open, h->proj_out.as<double2>(), h->nrhs, h->stream));
    return IOBM_OK;
}

int run_batch(iobm_handle* h) {
    if (h->nrhs == 0) {
        h->solved = true;
        h->hstate.clear();
        return IOBM_OK;
    }
    int rc = bind_workspace(h, h->nrhs);
    if (rc) return rc;
    rc = (h->opt.precision == IOBM_MIXED) ? run_solver<float>(h, h->nrhs)
                                          : run_solver<double>(h, h->nrhs);
    if (rc) return rc;
    if (h->opt.precision == IOBM_MIXED) {
        rc = escalate_fp64(h);
        if (rc) return rc;
    }
    rc = launch_projections(h);
    if (rc) return rc;
    h->solved = true;
    return IOBM_OK;
}

// ---- several junctions in one graph ------------------------------------------

// Capture the body of a junction's WHILE node: one chunk of its iterations and
// the kernel that sets the loop condition.
template <typename T>
int capture_batch_body(iobm_handle* h, cudaGraph_t body, cudaGraphConditionalHandle cond,
                       long long& per_chunk) {
    CK(cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    int rc = launch_chunk<T>(h, h->nrhs, false, per_chunk);
    if (rc == IOBM_OK) {
        const int max_chunks = iter_cap(h) / chunk_length(h) + 4;
        const cudaError_t e = launch_batch_cond(cond, h->st, h->nrhs, h->batch_ctr.as<int>(),
                                                max_chunks, h->stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "batch loop condition");
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(h, e, "batch body capture");
    return IOBM_OK;
}

// Solve every junction of the batch: per-junction set-up and start on each
// handle's stream, then ONE graph launch holding a WHILE node per junction
// (its chunk of COCG iterations repeated on the device until the junction's
// RHS have all stopped), then the per-junction ends and projections.
int solve_batch(int n, iobm_handle* const* hs, const double* const* E, const int* nE, int side) {
    std::vector<long long> launches(n, 0), per_chunk(n, 0);
    std::vector<int> active;
    for (int j = 0; j < n; ++j) {
        iobm_handle* h = hs[j];
        h->solved = false;
        int rc = prepare_rhs(h, E[j], nE[j], nullptr, 0, side, 0);
        if (rc) return rc;
        if (h->nrhs == 0) {
            h->solved = true;
            h->hstate.clear();
            continue;
        }
        rc = bind_workspace(h, h->nrhs);
        if (rc) return rc;
        CK(h->batch_ctr.ensure(sizeof(int)));
        CK(cudaMemsetAsync(h->batch_ctr.p, 0, sizeof(int), h->stream));
        rc = (h->opt.precision == IOBM_MIXED) ? solver_prologue<float>(h, h->nrhs, launches[j])
                                              : solver_prologue<double>(h, h->nrhs, launches[j]);
        if (rc) return rc;
        active.push_back(j);
    }
    if (active.empty()) return IOBM_OK;
    iobm_handle* h0 = hs[active[0]];
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (done) cudaEventDestroy(done);
    };
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(h0, e, "batch graph set-up");
    }
    for (int j : active) {
        iobm_handle* h = hs[j];
        cudaGraphConditionalHandle cond;
        e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = cond;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(h, e, "batch WHILE node");
        }
        const int rc = (h->opt.precision == IOBM_MIXED)
                           ? capture_batch_body<float>(h, p.conditional.phGraph_out[0], cond, per_chunk[j])
                           : capture_batch_body<double>(h, p.conditional.phGraph_out[0], cond, per_chunk[j]);
        if (rc) {
            cleanup();
            return rc;
        }
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    // the graph starts when every junction's start has finished, and every
    // junction's end waits for the graph
    for (int j : active) {
        if (e == cudaSuccess) e = cudaEventRecord(hs[j]->ev_sync, hs[j]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h0->stream, hs[j]->ev_sync, 0);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, h0->stream);
    if (e == cudaSuccess) e = cudaEventRecord(done, h0->stream);
    for (int j : active)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hs[j]->stream, done, 0);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(h0, e, "batch graph launch");
    }
    int first_rc = IOBM_OK;
    for (int j : active) {
        iobm_handle* h = hs[j];
        int chunks = 0;
        e = cudaMemcpyAsync(&chunks, h->batch_ctr.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        int rc = (e == cudaSuccess) ? IOBM_OK : cuda_fail(h, e, "batch chunk count");
        launches[j] += (long long)chunks * (per_chunk[j] + 1);
        if (!rc)
            rc = (h->opt.precision == IOBM_MIXED) ? solver_epilogue<float>(h, h->nrhs, launches[j])
                                                  : solver_epilogue<double>(h, h->nrhs, launches[j]);
        if (!rc && h->opt.precision == IOBM_MIXED) rc = escalate_fp64(h);
        if (!rc) rc = launch_projections(h);
        if (!rc) h->solved = true;
        if (rc && !first_rc) first_rc = rc;
    }
    cleanup();
    return first_rc;
}

// t and r of every incident channel (host, FP64): combine the projection sums
// of its real-profile solves, subtract the unit incident wave on the entry
// planes, and apply the N_f x N_f projection row (Eq. 6).
int compute_tr(iobm_handle* h, std::vector<std::complex<double>>& t,
               std::vector<std::complex<double>>& r) {
    using cdd = std::complex<double>;
    const int nf = h->nf;
    const int mo = std::max(h->max_open, 1);
    std::vector<double2> out((size_t)std::max(h->nrhs, 1) * mo * 2 * kMaxNf);
    if (h->nrhs > 0) {
        CK(cudaMemcpyAsync(out.data(), h->proj_out.p, sizeof(double2) * (size_t)h->nrhs * mo * 2 * kMaxNf,
                           cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    const int nu = (int)h->users.size();
    t.assign((size_t)std::max(nu, 1) * mo, 0.0);
    r.assign((size_t)std::max(nu, 1) * mo, 0.0);
    auto S = [&](int internal, int o, int side, int d) {
        const double2 v = out[(((size_t)internal * mo + o) * 2 + side) * kMaxNf + d];
        return cdd(v.x, v.y);
    };
    for (int i = 0; i < nu; ++i) {
        const iobm_handle::User& U = h->users[i];
        const ModeTables& mt = h->energies[U.energy];
        const cdd ci = cdd(0.0, (double)U.sign);
        for (int o = 0; o < mt.nopen; ++o) {
            cdd tt = 0.0, rr = 0.0;
            for (int d = 0; d < nf; ++d) {
                cdd se = S(U.ic, o, 1 - U.side, d), sn = S(U.ic, o, U.side, d);
                if (U.is >= 0) {
                    se += ci * S(U.is, o, 1 - U.side, d);
                    sn += ci * S(U.is, o, U.side, d);
                }
                if (o == U.chan) sn -= std::pow(mt.lam_in[U.chan], d);
                tt += mt.mrow[(size_t)o * nf + d] * se;
                rr += mt.mrow[(size_t)o * nf + d] * sn;
            }
            t[(size_t)i * mo + o] = tt;
            r[(size_t)i * mo + o] = rr;
        }
    }
    return IOBM_OK;
}

int status_of_internal(const RhsState& S) {
    switch (S.status) {
        case ST_CONVERGED: return IOBM_OK;
        case ST_BREAKDOWN: return IOBM_E_BREAKDOWN;
        default: return IOBM_E_NOCONV;
    }
}

}  // namespace

// ============================================================================
// Time the fused COCG stencil (p = z + beta p_old, A p, p^T A p) on nrhs RHS of
// this grid for every candidate z-chunk and stencil kernel, keep the fastest.
template <typename T>
int autotune_stencil(iobm_handle* h, int nrhs, int* zchunk_out, int* variant_out) {
    using C = typename Cplx<T>::type;
    int rc = bind_workspace(h, nrhs);
    if (rc) return rc;
    const size_t bytes = sizeof(C) * (size_t)nrhs * h->npts;
    CK(cudaMemsetAsync(h->vz, 0, bytes, h->stream));
    CK(cudaMemsetAsync(h->vp[0], 0, bytes, h->stream));
    StencilArgs<T> a = op_args<T>(h);
    a.x = (const C*)h->vz;
    a.pbufs[0] = (C*)h->vp[0];
    a.pbufs[1] = (C*)h->vp[1];
    a.y = (C*)h->vq;
    a.fused_p = 1;
    a.state = nullptr;   // every RHS active, beta = 0
    a.dot_mode = 1;
    a.dot_part = h->mu_part;
    a.slot_stride = h->slot_stride;
    const int zcands[3] = {kZChunkMin, 32, 64};
    // FP32: the fastest kernel for the shape, the register-pipelined rows, the one-row
    // bulk-copy rows, the shared-memory plane ring; FP64: one kernel
    const int vcands[4] = {0, 1, 3, 4};
    const int nvar = std::is_same<T, float>::value ? 4 : 1;
    float best = -1.f;
    int best_z = h->zchunk, best_v = h->stencil_variant;
    for (int zi = 0; zi < 3; ++zi) {
        const int zc = zcands[zi];
        if (zi > 0 && zcands[zi - 1] >= h->g.nz) break;   // larger chunks are all the same launch
        for (int vi = 0; vi < nvar; ++vi) {
            const int v = vcands[vi];
            a.zchunk = zc;
            a.variant = v;
            CK(launch_stencil<T>(a, nrhs, h->stream));   // warm-up
            CK(cudaEventRecord(h->ev_t0, h->stream));
            for (int r = 0; r < 3; ++r) CK(launch_stencil<T>(a, nrhs, h->stream));
            CK(cudaEventRecord(h->ev_t1, h->stream));
            CK(cudaEventSynchronize(h->ev_t1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1));
            if (best < 0.f || ms < best) {
                best = ms;
                best_z = zc;
                best_v = v;
            }
        }
    }
    h->zchunk = best_z;
    h->stencil_variant = best_v;
    rc = bind_workspace(h, nrhs);   // slot counts follow the chosen z-chunk
    if (rc) return rc;
    rc = check_err_flag(h);
    if (rc) return rc;
    if (zchunk_out) *zchunk_out = best_z;
    if (variant_out) *variant_out = best_v;
    return IOBM_OK;
}

// Average CUDA-event time of the fused COCG operator launch (p = z + beta p_old,
// q = (E - T - V) p, p^T q partials) on nrhs RHS with every RHS active, with the
// handle's tiling: one warm-up launch, then reps timed launches.
template <typename T>
int time_operator(iobm_handle* h, int nrhs, int reps, double* ms_out) {
    using C = typename Cplx<T>::type;
    int rc = bind_workspace(h, nrhs);
    if (rc) return rc;
    const size_t bytes = sizeof(C) * (size_t)nrhs * h->npts;
    // nonzero operands (every float 0x3c3c3c3c, about 0.0115)
    CK(cudaMemsetAsync(h->vz, 0x3c, bytes, h->stream));
    CK(cudaMemsetAsync(h->vp[0], 0x3c, bytes, h->stream));
    StencilArgs<T> a = op_args<T>(h);
    a.x = (const C*)h->vz;
    a.pbufs[0] = (C*)h->vp[0];
    a.pbufs[1] = (C*)h->vp[1];
    a.y = (C*)h->vq;
    a.fused_p = 1;
    a.state = nullptr;   // every RHS active
    a.dot_mode = 1;
    a.dot_part = h->mu_part;
    a.slot_stride = h->slot_stride;
    CK(launch_stencil<T>(a, nrhs, h->stream));   // warm-up
    CK(cudaEventRecord(h->ev_t0, h->stream));
    for (int r = 0; r < reps; ++r) CK(launch_stencil<T>(a, nrhs, h->stream));
    CK(cudaEventRecord(h->ev_t1, h->stream));
    CK(cudaEventSynchronize(h->ev_t1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1));
    *ms_out = ms / reps;
    return check_err_flag(h);
}

extern "C" {

int iobm_time_operator(iobm_handle* h, int nrhs, int reps, double* ms_per_launch) {
    if (!h || nrhs < 1 || reps < 1 || !ms_per_launch)
        return h ? fail(h, IOBM_E_ARG, "time_operator needs nrhs >= 1, reps >= 1") : IOBM_E_ARG;
    if (cudaEventRecord(h->ev_sync, h->user_stream) == cudaSuccess)
        cudaStreamWaitEvent(h->stream, h->ev_sync, 0);
    const int rc = (h->opt.precision == IOBM_MIXED) ? time_operator<float>(h, nrhs, reps, ms_per_launch)
                                                    : time_operator<double>(h, nrhs, reps, ms_per_launch);
    h->solved = false;
    return rc;
}

void iobm_default_options(iobm_options* o) {
    if (!o) return;
    o->alpha = 1.8;
    o->use_precond = IOBM_PRECOND_FOURIER;
    o->tol = 1e-8;
    o->max_iter = 20000;
    o->precision = IOBM_MIXED;
    o->refine_delta = 0.01;
    o->chunk = 32;
    o->max_iter_mixed = 1000;
    o->op_form = IOBM_OP_AUTO;
    o->fp64_modes = -1;
    o->sigma_form = IOBM_SIGMA_FFT;
}

const char* iobm_status_string(int s) {
    switch (s) {
        case IOBM_OK: return "ok";
        case IOBM_E_ARG: return "invalid argument";
        case IOBM_E_THRESHOLD: return "energy at a channel threshold";
        case IOBM_E_PROJ_BOUNDARY: return "projector touches the self-energy planes";
        case IOBM_E_NOCONV: return "not converged";
        case IOBM_E_BREAKDOWN: return "COCG breakdown";
        case IOBM_E_TIMEOUT: return "device wait timed out";
        case IOBM_E_CUDA: return "CUDA error";
        case IOBM_E_STATE: return "call out of order";
        case IOBM_E_UNSUPPORTED: return "unsupported size";
        default: return "unknown status";
    }
}

const char* iobm_last_error(const iobm_handle* h) { return h ? h->err.c_str() : "null handle"; }

double iobm_fermi_energy(const iobm_handle* h) {
    if (!h) return 0.0;
    return std::pow(9.0 * M_PI / 4.0, 2.0 / 3.0) / (2.0 * h->rs * h->rs);
}

int iobm_create(const iobm_grid* grid, const double* V_loc, const iobm_projectors* proj, double rs,
                const iobm_options* opts, void* cuda_stream, iobm_handle** out) {
    if (!out) return IOBM_E_ARG;
    *out = nullptr;
    if (!grid || !V_loc) return IOBM_E_ARG;
    iobm_handle* h = new iobm_handle();
    h->g = *grid;
    h->nf = grid->nf;
    h->rs = rs;
    iobm_default_options(&h->opt);
    if (opts) h->opt = *opts;
    auto bad = [&](int code, const std::string& m) {
        h->err = m;
        *out = h;   // returned so that iobm_last_error can be read; caller destroys
        return code;
    };
    const iobm_grid& g = h->g;
    if (g.nx < 1 || g.ny < 1 || g.nf < 1 || g.nf > kMaxNf || g.nz < 2 * g.nf + 1 ||
        !(g.hx > 0) || !(g.hy > 0) || !(g.hz > 0))
        return bad(IOBM_E_ARG, "grid sizes or spacings out of range (need nf in 1..4, nz >= 2 nf + 1)");
    if (!(rs > 0)) return bad(IOBM_E_ARG, "rs must be positive");
    if (!(h->opt.tol > 0) || h->opt.max_iter < 1 || h->opt.max_iter_mixed < 1 ||
        !(h->opt.refine_delta > 0 && h->opt.refine_delta < 1) ||
        (h->opt.precision != IOBM_FP64 && h->opt.precision != IOBM_MIXED) || !(h->opt.alpha > 0) ||
        h->opt.use_precond < IOBM_PRECOND_NONE || h->opt.use_precond > IOBM_PRECOND_EQ10_FOURIER ||
        (h->opt.op_form != IOBM_OP_AUTO && h->opt.op_form != IOBM_OP_EXPLICIT) ||
        h->opt.fp64_modes < -1 ||
        (h->opt.sigma_form != IOBM_SIGMA_FFT && h->opt.sigma_form != IOBM_SIGMA_DENSE))
        return bad(IOBM_E_ARG, "invalid solver options");
    h->nxy = g.nx * g.ny;
    h->npts = (long long)h->nxy * g.nz;
    if (h->npts > (1LL << 31) - 1) return bad(IOBM_E_UNSUPPORTED, "grid larger than 2^31 points");
    if (h->nxy > kSmemPlaneLimit && !large_plane_supported(g.nx, g.ny))
        return bad(IOBM_E_UNSUPPORTED, "lateral sizes above 256 are not supported");
    if (g.nz < 2 * g.nf + 2)
        return bad(IOBM_E_ARG, "need at least 2 nf + 2 planes");
    std::vector<int> rx, ry;
    if (!fft_plan(g.nx, rx) || !fft_plan(g.ny, ry))
        return bad(IOBM_E_UNSUPPORTED, "lateral sizes may only have the prime factors 2, 3 and 5");
    if ((int)rx.size() > kMaxRadixPasses || (int)ry.size() > kMaxRadixPasses)
        return bad(IOBM_E_UNSUPPORTED, "too many FFT passes");
    h->ax.n = g.nx;
    h->ax.npass = (int)rx.size();
    for (size_t i = 0; i < rx.size(); ++i) h->ax.radix[i] = rx[i];
    h->ay.n = g.ny;
    h->ay.npass = (int)ry.size();
    for (size_t i = 0; i < ry.size(); ++i) h->ay.radix[i] = ry[i];
    for (long long i = 0; i < h->npts; ++i)
        if (!std::isfinite(V_loc[i])) return bad(IOBM_E_ARG, "non-finite V_loc");
    std::string msg;
    int rc = build_projectors(proj ? proj->nproj : 0, proj ? proj->row_ptr : nullptr,
                              proj ? proj->idx : nullptr, proj ? proj->val : nullptr,
                              proj ? proj->coupling : nullptr, g.nx, g.ny, g.nz, g.nf, h->pt, msg);
    if (rc) return bad(rc, msg);
    h->w = fd_weights(g.nf);

    h->user_stream = (cudaStream_t)cuda_stream;
    if (const char* env = std::getenv("IOBM_GRAPH_CONDITIONALS"))
        h->graph_conditionals = std::strcmp(env, "0") != 0;
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cond_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cond_side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_zfork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_zjoin, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_sfork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_sjoin, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_sync, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev_t0);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev_t1);
    if (e == cudaSuccess) e = sigma_prepare();
    if (e == cudaSuccess) e = precond_prepare();
    if (e == cudaSuccess) e = stencil_prepare();
    if (e == cudaSuccess) e = fft_large_prepare();
    if (e != cudaSuccess) return bad(IOBM_E_CUDA, std::string("stream/event setup: ") + cudaGetErrorString(e));

    std::vector<float> v32(h->npts);
    std::vector<double> v64(V_loc, V_loc + h->npts);
    for (long long i = 0; i < h->npts; ++i) v32[i] = (float)V_loc[i];
    auto tw = [](int n, double sign, std::vector<double2>& t64, std::vector<float2>& t32) {
        t64.resize(n);
        t32.resize(n);
        for (int k = 0; k < n; ++k) {
            const double a = sign * 2.0 * M_PI * k / n;
            t64[k] = make_double2(std::cos(a), std::sin(a));
            t32[k] = make_float2((float)t64[k].x, (float)t64[k].y);
        }
    };
    std::vector<double2> tx64, ty64, px64, py64;
    std::vector<float2> tx32, ty32, px32, py32;
    tw(g.nx, -1.0, tx64, tx32);
    tw(g.ny, -1.0, ty64, ty32);
    tw(g.nx, +1.0, px64, px32);
    tw(g.ny, +1.0, py64, py32);
    std::vector<float> pv32(h->pt.pval.begin(), h->pt.pval.end());
    std::vector<float> uv32(h->pt.uval.begin(), h->pt.uval.end());
    // union-of-supports points of plane k: uidx[uplane[k] .. uplane[k+1]) (uidx is sorted)
    std::vector<int> uplane(g.nz + 1);
    for (int k = 0; k <= g.nz; ++k)
        uplane[k] = (int)(std::lower_bound(h->pt.uidx.begin(), h->pt.uidx.end(),
                                           (long long)k * h->nxy) - h->pt.uidx.begin());
    cudaStream_t s = h->stream;
    if ((e = upload(h->V32, v32, s)) || (e = upload(h->V64, v64, s)) || (e = upload(h->twx32, tx32, s)) ||
        (e = upload(h->twy32, ty32, s)) || (e = upload(h->twx64, tx64, s)) ||
        (e = upload(h->twy64, ty64, s)) || (e = upload(h->phx, px64, s)) || (e = upload(h->phy, py64, s)) ||
        (e = upload(h->pptr, h->pt.pptr, s)) || (e = upload(h->pidx, h->pt.pidx, s)) ||
        (e = upload(h->pval32, pv32, s)) || (e = upload(h->pval64, h->pt.pval, s)) ||
        (e = upload(h->pcoup, h->pt.coupling, s)) || (e = upload(h->uidx, h->pt.uidx, s)) ||
        (e = upload(h->uptr, h->pt.uptr, s)) || (e = upload(h->uproj, h->pt.uproj, s)) ||
        (e = upload(h->uval32, uv32, s)) || (e = upload(h->uval64, h->pt.uval, s)) ||
        (e = upload(h->uplane, uplane, s)) ||
        (e = h->errflag.ensure(sizeof(int))) || (e = cudaMemsetAsync(h->errflag.p, 0, sizeof(int), s)))
        return bad(IOBM_E_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bad(IOBM_E_CUDA, std::string("create: ") + cudaGetErrorString(e));
    *out = h;
    return IOBM_OK;
}

int iobm_create_batch(int n, const iobm_grid* grids, const double* const* V,
                      const iobm_projectors* projs, const double* rs, const iobm_options* opts,
                      void* cuda_stream, iobm_handle** out) {
    if (n < 1 || !grids || !V || !rs || !out) return IOBM_E_ARG;
    for (int j = 0; j < n; ++j) out[j] = nullptr;
    for (int j = 0; j < n; ++j) {
        const iobm_projectors* pj = (projs && projs[j].nproj > 0) ? &projs[j] : nullptr;
        const int rc = iobm_create(&grids[j], V[j], pj, rs[j], opts, cuda_stream, &out[j]);
        if (rc) {
            for (int i = 0; i < j; ++i) {
                iobm_destroy(out[i]);
                out[i] = nullptr;
            }
            out[j] = nullptr;
            return rc;
        }
    }
    return IOBM_OK;
}

void iobm_destroy(iobm_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->chunk_exec) cudaGraphExecDestroy(h->chunk_exec);
    if (h->pin) cudaFreeHost(h->pin);
    DevBuf* bufs[] = {&h->V32, &h->V64, &h->twx32, &h->twy32, &h->twx64, &h->twy64, &h->phx,
                      &h->phy, &h->pptr, &h->pidx, &h->pval32, &h->pval64, &h->pcoup, &h->uidx,
                      &h->uptr, &h->uproj, &h->uval32, &h->uval64, &h->sig32, &h->sig64, &h->pc32,
                      &h->pc64, &h->ediag, &h->rhs_energy, &h->descs, &h->open_ptr, &h->open_bins,
                      &h->proj_out, &h->apply_sig32, &h->apply_sig64, &h->apply_pc32,
                      &h->apply_pc64, &h->apply_ediag, &h->ws_owned, &h->errflag,
                      &h->batch_ctr, &h->sig_scratch, &h->sig_end, &h->kb_scratch, &h->uplane, &h->esc_ws,
                      &h->esc_descs, &h->esc_rhs_energy, &h->rhs_sign, &h->apply_sign,
                      &h->gph32, &h->gph64, &h->gpx, &h->gpy, &h->esc_rhs_sign,
                      &h->zflag, &h->zf_bins, &h->zf_pc, &h->zf_tab, &h->zf_scr,
                      &h->dense32, &h->dense64,
                      &h->apply_dense32, &h->apply_dense64, &h->dense_k, &h->dense_part};
    for (DevBuf* b : bufs) b->release();
    if (h->ev_sync) cudaEventDestroy(h->ev_sync);
    if (h->ev_t0) cudaEventDestroy(h->ev_t0);
    if (h->ev_t1) cudaEventDestroy(h->ev_t1);
    for (cudaEvent_t ev : h->kev) cudaEventDestroy(ev);
    if (h->stream) cudaStreamDestroy(h->stream);
    if (h->cond_stream) cudaStreamDestroy(h->cond_stream);
    if (h->side_stream) cudaStreamDestroy(h->side_stream);
    if (h->cond_side) cudaStreamDestroy(h->cond_side);
    if (h->ev_zfork) cudaEventDestroy(h->ev_zfork);
    if (h->ev_zjoin) cudaEventDestroy(h->ev_zjoin);
    if (h->ev_sfork) cudaEventDestroy(h->ev_sfork);
    if (h->ev_sjoin) cudaEventDestroy(h->ev_sjoin);
    delete h;
}

int iobm_open_channels(iobm_handle* h, double E, int* n_open, int max_out, int* nu, double* vel) {
    if (!h || !n_open) return IOBM_E_ARG;
    ModeTables mt;
    std::string msg;
    const int rc = build_mode_tables(h->g.nx, h->g.ny, h->g.hx, h->g.hy, h->g.hz, h->nf, E, false, mt,
                                     msg, h->kappa[0], h->kappa[1]);
    if (rc) return fail(h, rc == 2 ? IOBM_E_THRESHOLD : IOBM_E_UNSUPPORTED, msg);
    *n_open = mt.nopen;
    for (int c = 0; c < mt.nopen && c < max_out; ++c) {
        if (nu) {
            nu[2 * c] = mt.open_nux[c];
            nu[2 * c + 1] = mt.open_nuy[c];
        }
        if (vel) vel[c] = mt.vel[c];
    }
    return IOBM_OK;
}

int iobm_workspace_size(iobm_handle* h, int nrhs, size_t* bytes) {
    if (!h || !bytes || nrhs < 0) return IOBM_E_ARG;
    *bytes = workspace_bytes(h, nrhs, h->opt.precision);
    return IOBM_OK;
}

int iobm_set_workspace(iobm_handle* h, void* dev_ptr, size_t bytes) {
    if (!h) return IOBM_E_ARG;
    if (dev_ptr && (reinterpret_cast<uintptr_t>(dev_ptr) & 255))
        return fail(h, IOBM_E_ARG, "workspace must be 256-byte aligned");
    h->ws = dev_ptr;
    h->ws_bytes = dev_ptr ? bytes : 0;
    h->solved = false;
    return IOBM_OK;
}

int iobm_solve(iobm_handle* h, const double* E, int nE, const int* channels, int nch, int side) {
    if (!h || !E || nE < 1 || (channels && nch < 0) || (side != 0 && side != 1))
        return h ? fail(h, IOBM_E_ARG, "invalid solve arguments") : IOBM_E_ARG;
    h->solved = false;
    // order after the caller's stream
    if (cudaEventRecord(h->ev_sync, h->user_stream) == cudaSuccess)
        cudaStreamWaitEvent(h->stream, h->ev_sync, 0);
    int rc = prepare_rhs(h, E, nE, channels, nch, side, 0);
    if (rc) return rc;
    rc = run_batch(h);
    if (rc) return rc;
    CK(cudaEventRecord(h->ev_sync, h->stream));
    CK(cudaStreamWaitEvent(h->user_stream, h->ev_sync, 0));
    return IOBM_OK;
}

int iobm_autotune(iobm_handle* h, int nrhs, int* zchunk, int* variant) {
    if (!h || nrhs < 1) return h ? fail(h, IOBM_E_ARG, "autotune needs nrhs >= 1") : IOBM_E_ARG;
    return (h->opt.precision == IOBM_MIXED) ? autotune_stencil<float>(h, nrhs, zchunk, variant)
                                            : autotune_stencil<double>(h, nrhs, zchunk, variant);
}

int iobm_set_tiling(iobm_handle* h, int zchunk, int variant) {
    if (!h) return IOBM_E_ARG;
    if (zchunk < kZChunkMin || (variant != 0 && variant != 1 && variant != 3 && variant != 4))
        return fail(h, IOBM_E_ARG, "z-chunk below the minimum or unknown stencil variant");
    h->zchunk = zchunk;
    h->stencil_variant = variant;
    return IOBM_OK;
}

int iobm_solve_batch(int n, iobm_handle* const* handles, const double* const* E, const int* nE,
                     int side) {
    if (n < 1 || !handles || !E || !nE || (side != 0 && side != 1)) return IOBM_E_ARG;
    for (int j = 0; j < n; ++j) {
        if (!handles[j] || !E[j] || nE[j] < 1) return IOBM_E_ARG;
        if (bloch(handles[j]))
            return fail(handles[j], IOBM_E_UNSUPPORTED, "batched solves run at a zero Bloch vector");
        if (dense_sigma(handles[j]))
            return fail(handles[j], IOBM_E_UNSUPPORTED, "batched solves use the FFT self-energy");
        for (int i = 0; i < j; ++i)
            if (handles[i] == handles[j]) return fail(handles[j], IOBM_E_ARG, "a handle appears twice in the batch");
    }
    return solve_batch(n, handles, E, nE, side);
}

int iobm_eigenchannels(iobm_handle* h, int e, double* tau, int max_out, int* n_out) {
    if (!h || !n_out) return IOBM_E_ARG;
    if (!h->solved) return fail(h, IOBM_E_STATE, "no solve to report on");
    if (e < 0 || e >= (int)h->energies.size()) return fail(h, IOBM_E_ARG, "energy index out of range");
    const ModeTables& mt = h->energies[e];
    const int n = mt.nopen;
    *n_out = n;
    if (!tau) return IOBM_OK;
    if (max_out < n) return fail(h, IOBM_E_ARG, "max_out is smaller than the open-channel count");
    if (n == 0) return IOBM_OK;
    // the flux-normalised transmission matrix tt[o][c] = t_oc sqrt(v_o / v_c) needs
    // every open incident channel of this energy from one side
    std::vector<int> user_of(n, -1);
    for (size_t i = 0; i < h->users.size(); ++i)
        if (h->users[i].energy == e) user_of[h->users[i].chan] = (int)i;
    for (int c = 0; c < n; ++c)
        if (user_of[c] < 0) return fail(h, IOBM_E_STATE, "eigenchannels need every open incident channel");
    std::vector<std::complex<double>> t, r;
    const int rc = compute_tr(h, t, r);
    if (rc) return rc;
    const int mo = std::max(h->max_open, 1);
    std::vector<std::complex<double>> tt((size_t)n * n);
    for (int c = 0; c < n; ++c)
        for (int o = 0; o < n; ++o)
            tt[(size_t)o * n + c] = t[(size_t)user_of[c] * mo + o] * std::sqrt(mt.vel[o] / mt.vel[c]);
    // T^dagger T (Hermitian, positive semidefinite)
    std::vector<std::complex<double>> m((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            std::complex<double> acc = 0.0;
            for (int o = 0; o < n; ++o) acc += std::conj(tt[(size_t)o * n + i]) * tt[(size_t)o * n + j];
            m[(size_t)i * n + j] = acc;
            m[(size_t)j * n + i] = std::conj(acc);
        }
    std::vector<double> w;
    hermitian_eigenvalues(m, n, w);
    for (int i = 0; i < n; ++i) tau[i] = w[i];
    return IOBM_OK;
}

int iobm_num_rhs(const iobm_handle* h) { return h ? (int)h->users.size() : 0; }

int iobm_max_open(const iobm_handle* h) { return (h && h->solved) ? h->max_open : 0; }

int iobm_solve_rhs_count(iobm_handle* h, const double* E, int nE, const int* channels, int nch,
                         int* n_internal) {
    if (!h || !E || nE < 1 || !n_internal) return IOBM_E_ARG;
    const int rc = prepare_rhs(h, E, nE, channels, nch, 0, 0, false);
    h->solved = false;
    if (rc) return rc;
    *n_internal = h->nrhs;
    return IOBM_OK;
}

int iobm_transmission(iobm_handle* h, double* T, double* R, int max_open, double* G, int* nopen,
                      iobm_report* reports) {
    if (!h) return IOBM_E_ARG;
    if (!h->solved) return fail(h, IOBM_E_STATE, "no solve to report on");
    if ((T || R) && max_open < h->max_open)
        return fail(h, IOBM_E_ARG, "max_open is smaller than the largest open-channel count");
    std::vector<std::complex<double>> t, r;
    const int rc = compute_tr(h, t, r);
    if (rc) return rc;
    const int mo = std::max(h->max_open, 1);
    const int nE = (int)h->energies.size();
    if (G)
        for (int e = 0; e < nE; ++e) G[e] = 0.0;
    if (nopen)
        for (int e = 0; e < nE; ++e) nopen[e] = h->energies[e].nopen;
    for (size_t i = 0; i < h->users.size(); ++i) {
        const iobm_handle::User& U = h->users[i];
        const ModeTables& mt = h->energies[U.energy];
        const double vin = mt.vel[U.chan];
        for (int o = 0; o < max_open && (T || R); ++o) {
            double Tv = 0.0, Rv = 0.0;
            if (o < mt.nopen) {
                Tv = std::norm(t[i * mo + o]) * mt.vel[o] / vin;
                Rv = std::norm(r[i * mo + o]) * mt.vel[o] / vin;
            }
            if (T) T[i * max_open + o] = Tv;
            if (R) R[i * max_open + o] = Rv;
        }
        if (G)
            for (int o = 0; o < mt.nopen; ++o) G[U.energy] += std::norm(t[i * mo + o]) * mt.vel[o] / vin;
        if (reports) {
            const RhsState& Sc = h->hstate[U.ic];
            iobm_report& rp = reports[i];
            rp.energy_index = U.energy;
            rp.channel = U.chan;
            rp.side = U.side;
            rp.status = status_of_internal(Sc);
            rp.iterations = Sc.iters;
            rp.replacements = Sc.replacements;
            double num = Sc.res64 * std::sqrt(Sc.bb), den = Sc.bb;
            if (U.is >= 0) {
                const RhsState& Ss = h->hstate[U.is];
                if (rp.status == IOBM_OK) rp.status = status_of_internal(Ss);
                rp.iterations = std::max(rp.iterations, Ss.iters);
                rp.replacements = std::max(rp.replacements, Ss.replacements);
                num += Ss.res64 * std::sqrt(Ss.bb);
                den += Ss.bb;
            }
            rp.residual = den > 0 ? num / std::sqrt(den) : 0.0;   // bound on ||b - A psi|| / ||b||
        }
    }
    return IOBM_OK;
}

int iobm_solution(iobm_handle* h, int rhs, void* dst, int dst_is_device) {
    if (!h || !dst) return IOBM_E_ARG;
    if (!h->solved || rhs < 0 || rhs >= (int)h->users.size())
        return fail(h, IOBM_E_STATE, "no such solved incident channel");
    const iobm_handle::User& U = h->users[rhs];
    const size_t bytes = sizeof(double2) * h->npts;
    double2* tmp = h->y64;   // scratch of the last solve
    if (bloch(h)) {
        // psi = exp(i s kappa.r) phi, s = -1 for the -kappa channels (the upper slots)
        const int sgn = U.energy < (int)h->energies.size() / 2 ? 1 : -1;
        CK(launch_gauge(tmp, h->x64 + (size_t)U.ic * h->npts, h->gpx.as<double2>(),
                        h->gpy.as<double2>(), sgn, h->g.nx, h->g.ny, h->g.nz, h->stream));
    } else {
        CK(launch_combine(tmp, h->x64 + (size_t)U.ic * h->npts, make_double2(1.0, 0.0),
                          U.is >= 0 ? h->x64 + (size_t)U.is * h->npts : nullptr,
                          make_double2(0.0, (double)U.sign), h->npts, h->stream));
    }
    CK(cudaMemcpyAsync(dst, tmp, bytes, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return IOBM_OK;
}

int iobm_grad_V(iobm_handle* h, double E, double* dGdV, int dst_is_device, double* G_out) {
    using cdd = std::complex<double>;
    if (!h || !dGdV) return IOBM_E_ARG;
    if (cudaEventRecord(h->ev_sync, h->user_stream) == cudaSuccess)
        cudaStreamWaitEvent(h->stream, h->ev_sync, 0);
    int rc = prepare_rhs(h, &E, 1, nullptr, 0, 0, 1);
    if (rc) return rc;
    const ModeTables& mt = h->energies[0];
    const int n = mt.nopen;
    // forward internal RHS come first; count them
    int nX = 0;
    for (const iobm_handle::User& U : h->users) nX = std::max(nX, std::max(U.ic, U.is) + 1);
    const int nY = h->nrhs - nX;
    rc = run_batch(h);
    if (rc) return rc;
    std::vector<cdd> t, r;
    rc = compute_tr(h, t, r);
    if (rc) return rc;
    const int mo = std::max(h->max_open, 1);
    // psi_i = sum_k B[i][k] X_k;  lambda_o = sum_j L[o][j] Y_j;  U = C B
    std::vector<cdd> B((size_t)std::max(n, 1) * std::max(nX, 1), 0.0), Lm((size_t)std::max(n, 1) * std::max(nY, 1), 0.0);
    for (int i = 0; i < n; ++i) {
        const iobm_handle::User& U = h->users[i];
        B[(size_t)i * nX + U.ic] = 1.0;
        if (U.is >= 0) B[(size_t)i * nX + U.is] = cdd(0.0, (double)U.sign);
        // adjoint of channel i: w ~ exp(-i G.r) = cos -+ i sin, the opposite sign
        const int jc = U.ic, js = U.is;   // the adjoint list mirrors the forward one
        Lm[(size_t)i * nY + jc] = 1.0;
        if (js >= 0) Lm[(size_t)i * nY + js] = cdd(0.0, -(double)U.sign);
    }
    double G = 0.0;
    std::vector<double2> Ud((size_t)std::max(n * nX, 1)), Ld((size_t)std::max(n * nY, 1));
    for (int o = 0; o < n; ++o) {
        for (int k = 0; k < nX; ++k) {
            cdd acc = 0.0;
            for (int i = 0; i < n; ++i) {
                const cdd toi = t[(size_t)i * mo + o];
                acc += (mt.vel[o] / mt.vel[i]) * std::conj(toi) * B[(size_t)i * nX + k];
            }
            Ud[(size_t)o * nX + k] = make_double2(acc.real(), acc.imag());
        }
        for (int j = 0; j < nY; ++j) Ld[(size_t)o * nY + j] = make_double2(Lm[(size_t)o * nY + j].real(), Lm[(size_t)o * nY + j].imag());
        for (int i = 0; i < n; ++i) G += std::norm(t[(size_t)i * mo + o]) * mt.vel[o] / mt.vel[i];
    }
    if (G_out) *G_out = G;
    DevBuf dU, dL, dg;
    CK(upload(dU, Ud, h->stream));
    CK(upload(dL, Ld, h->stream));
    double* gdev = dGdV;
    if (!dst_is_device) {
        CK(dg.ensure(sizeof(double) * h->npts));
        gdev = dg.as<double>();
    }
    if (n > 0) {
        CK(launch_gradient(h->x64, nX, h->x64 + (size_t)nX * h->npts, nY, dU.as<double2>(),
                           dL.as<double2>(), n, h->npts, gdev, h->stream));
    } else {
        CK(cudaMemsetAsync(gdev, 0, sizeof(double) * h->npts, h->stream));
    }
    if (!dst_is_device)
        CK(cudaMemcpyAsync(dGdV, gdev, sizeof(double) * h->npts, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    dU.release();
    dL.release();
    dg.release();
    CK(cudaEventRecord(h->ev_sync, h->stream));
    CK(cudaStreamWaitEvent(h->user_stream, h->ev_sync, 0));
    return IOBM_OK;
}

static int apply_common(iobm_handle* h, double E, int elem, const void* x, void* y, int nrhs,
                        bool precond) {
    if (!h || !x || !y || nrhs < 0 ||
        (elem != IOBM_ELEM_C64 && elem != IOBM_ELEM_C32 && !(elem == IOBM_ELEM_C64_DF && !precond)))
        return h ? fail(h, IOBM_E_ARG, "invalid apply arguments") : IOBM_E_ARG;
    if (nrhs == 0) return IOBM_OK;
    if (bloch(h) && !precond && elem == IOBM_ELEM_C32)
        return fail(h, IOBM_E_UNSUPPORTED, "the FP32 operator has no lateral Bloch phases");
    if (cudaEventRecord(h->ev_sync, h->user_stream) == cudaSuccess)
        cudaStreamWaitEvent(h->stream, h->ev_sync, 0);
    CK(ensure_sigma_scratch(h, nrhs));
    if (bloch(h)) {   // every vector at +kappa
        std::vector<int> ones(nrhs, 1);
        CK(upload(h->apply_sign, ones, h->stream));
    }
    long long launches = 0;
    const bool need_tables = !precond || h->opt.use_precond == IOBM_PRECOND_FOURIER;
    if (need_tables) {
        ModeTables mt;
        std::string msg;
        const int rc = build_mode_tables(h->g.nx, h->g.ny, h->g.hx, h->g.hy, h->g.hz, h->nf, E, true,
                                         mt, msg, h->kappa[0], h->kappa[1]);
        if (rc) return fail(h, rc == 2 ? IOBM_E_THRESHOLD : IOBM_E_UNSUPPORTED, msg);
        std::vector<double2> s64(mt.sigma.size()), p64(mt.pc.size());
        std::vector<float2> s32(mt.sigma.size()), p32(mt.pc.size());
        for (size_t i = 0; i < mt.sigma.size(); ++i) {
            s64[i] = make_double2(mt.sigma[i].real(), mt.sigma[i].imag());
            s32[i] = make_float2((float)s64[i].x, (float)s64[i].y);
        }
        for (size_t i = 0; i < mt.pc.size(); ++i) {
            p64[i] = make_double2(mt.pc[i].real(), mt.pc[i].imag());
            p32[i] = make_float2((float)p64[i].x, (float)p64[i].y);
        }
        std::vector<double> ed(1, E);
        CK(upload(h->apply_sig64, s64, h->stream));
        CK(upload(h->apply_sig32, s32, h->stream));
        if (dense_sigma(h) && !precond) {
            const int rc = build_dense_sigma(h, h->apply_sig64.p, 1, h->apply_dense32, h->apply_dense64);
            if (rc) return rc;
        }
        CK(upload(h->apply_pc64, p64, h->stream));
        CK(upload(h->apply_pc32, p32, h->stream));
        CK(upload(h->apply_ediag, ed, h->stream));
    }
    if (precond) {
        if (fourier_precond(h)) {
            if (elem == IOBM_ELEM_C64) {
                PrecondArgs<double> f = fourier_args<double>(h, h->apply_pc64.p);
                f.r = (const double2*)x;
                f.spec = (double2*)y;
                f.z = (double2*)y;
                CK(launch_precond_fourier<double>(f, nrhs, h->stream));
            } else {
                PrecondArgs<float> f = fourier_args<float>(h, h->apply_pc32.p);
                f.r = (const float2*)x;
                f.spec = (float2*)y;
                f.z = (float2*)y;
                CK(launch_precond_fourier<float>(f, nrhs, h->stream));
            }
        } else if (elem == IOBM_ELEM_C64) {
            StencilArgs<double> a = precond_args<double>(h);
            a.x = (const double2*)x;
            a.y = (double2*)y;
            CK(launch_stencil<double>(a, nrhs, h->stream));
        } else {
            StencilArgs<float> a = precond_args<float>(h);
            a.x = (const float2*)x;
            a.y = (float2*)y;
            CK(launch_stencil<float>(a, nrhs, h->stream));
        }
    } else {
        int rc2;
        if (elem == IOBM_ELEM_C64 || elem == IOBM_ELEM_C64_DF)
            rc2 = apply_operator<double>(h, x, y, nrhs, h->apply_sig64.p, h->apply_ediag.as<double>(),
                                         nullptr, nullptr, M_ALL, launches, elem == IOBM_ELEM_C64_DF,
                                         h->apply_sign.as<int>());
        else
            rc2 = apply_operator<float>(h, x, y, nrhs, h->apply_sig32.p, h->apply_ediag.as<double>(),
                                        nullptr, nullptr, M_ALL, launches);
        if (rc2) return rc2;
    }
    CK(cudaEventRecord(h->ev_sync, h->stream));
    CK(cudaStreamWaitEvent(h->user_stream, h->ev_sync, 0));
    CK(cudaStreamSynchronize(h->stream));
    return check_err_flag(h);
}

int iobm_apply(iobm_handle* h, double E, int elem, const void* x, void* y, int nrhs) {
    return apply_common(h, E, elem, x, y, nrhs, false);
}

int iobm_apply_precond(iobm_handle* h, double E, int elem, const void* x, void* y, int nrhs) {
    return apply_common(h, E, elem, x, y, nrhs, true);
}

int iobm_set_potential(iobm_handle* h, const double* V_loc, int src_is_device) {
    if (!h || !V_loc) return IOBM_E_ARG;
    std::vector<double> v64(h->npts);
    if (src_is_device) {
        CK(cudaMemcpy(v64.data(), V_loc, sizeof(double) * h->npts, cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(v64.data(), V_loc, sizeof(double) * h->npts);
    }
    for (long long i = 0; i < h->npts; ++i)
        if (!std::isfinite(v64[i])) return fail(h, IOBM_E_ARG, "non-finite V_loc");
    std::vector<float> v32(h->npts);
    for (long long i = 0; i < h->npts; ++i) v32[i] = (float)v64[i];
    CK(upload(h->V64, v64, h->stream));
    CK(upload(h->V32, v32, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->solved = false;
    return IOBM_OK;
}

int iobm_channels_host(const iobm_grid* g, double E, int* n_open, int max_out, int* nu,
                       double* vel, double* lam, double* btilde, double* mrow, double* sigma) {
    return iobm_channels_host_bloch(g, 0.0, 0.0, E, n_open, max_out, nu, vel, lam, btilde, mrow,
                                    sigma);
}

int iobm_channels_host_bloch(const iobm_grid* g, double kappa_x, double kappa_y, double E,
                             int* n_open, int max_out, int* nu, double* vel, double* lam,
                             double* btilde, double* mrow, double* sigma) {
    if (!g || !n_open || g->nx < 1 || g->ny < 1 || g->nf < 1 || g->nf > kMaxNf) return IOBM_E_ARG;
    if (!std::isfinite(kappa_x) || !std::isfinite(kappa_y)) return IOBM_E_ARG;
    ModeTables mt;
    std::string msg;
    const int rc = build_mode_tables(g->nx, g->ny, g->hx, g->hy, g->hz, g->nf, E, sigma != nullptr,
                                     mt, msg, kappa_x, kappa_y);
    if (rc) return rc == 2 ? IOBM_E_THRESHOLD : IOBM_E_UNSUPPORTED;
    const int nf = g->nf;
    *n_open = mt.nopen;
    for (int c = 0; c < mt.nopen && c < max_out; ++c) {
        if (nu) {
            nu[2 * c] = mt.open_nux[c];
            nu[2 * c + 1] = mt.open_nuy[c];
        }
        if (vel) vel[c] = mt.vel[c];
        if (lam) {
            lam[2 * c] = mt.lam_in[c].real();
            lam[2 * c + 1] = mt.lam_in[c].imag();
        }
        for (int d = 0; d < nf; ++d) {
            if (btilde) {
                btilde[2 * (c * nf + d)] = mt.btilde[(size_t)c * nf + d].real();
                btilde[2 * (c * nf + d) + 1] = mt.btilde[(size_t)c * nf + d].imag();
            }
            if (mrow) {
                mrow[2 * (c * nf + d)] = mt.mrow[(size_t)c * nf + d].real();
                mrow[2 * (c * nf + d) + 1] = mt.mrow[(size_t)c * nf + d].imag();
            }
        }
    }
    if (sigma)
        for (size_t i = 0; i < mt.sigma.size(); ++i) {
            sigma[2 * i] = mt.sigma[i].real();
            sigma[2 * i + 1] = mt.sigma[i].imag();
        }
    return IOBM_OK;
}

int iobm_set_bloch(iobm_handle* h, double kappa_x, double kappa_y) {
    if (!h) return IOBM_E_ARG;
    if (!std::isfinite(kappa_x) || !std::isfinite(kappa_y))
        return fail(h, IOBM_E_ARG, "non-finite Bloch vector");
    if ((kappa_x != 0.0 || kappa_y != 0.0) &&
        (h->opt.use_precond != IOBM_PRECOND_FOURIER || h->opt.op_form != IOBM_OP_AUTO ||
         dense_sigma(h)))
        return fail(h, IOBM_E_UNSUPPORTED,
                    "a nonzero Bloch vector needs the free-propagator preconditioner, the "
                    "implicit operator form and the FFT self-energy");
    h->kappa[0] = kappa_x;
    h->kappa[1] = kappa_y;
    h->solved = false;
    h->memo_E.clear();
    h->memo_tables.clear();
    if (!bloch(h)) return IOBM_OK;
    // exp(i kappa.r) on the lateral plane (KB gauge phases) and per axis (read-back)
    std::vector<double2> px(h->g.nx), py(h->g.ny), g64((size_t)h->nxy);
    std::vector<float2> g32((size_t)h->nxy);
    for (int x = 0; x < h->g.nx; ++x)
        px[x] = make_double2(std::cos(kappa_x * x * h->g.hx), std::sin(kappa_x * x * h->g.hx));
    for (int y = 0; y < h->g.ny; ++y)
        py[y] = make_double2(std::cos(kappa_y * y * h->g.hy), std::sin(kappa_y * y * h->g.hy));
    for (int y = 0; y < h->g.ny; ++y)
        for (int x = 0; x < h->g.nx; ++x) {
            const double a = kappa_x * x * h->g.hx + kappa_y * y * h->g.hy;
            g64[(size_t)y * h->g.nx + x] = make_double2(std::cos(a), std::sin(a));
            g32[(size_t)y * h->g.nx + x] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    CK(upload(h->gpx, px, h->stream));
    CK(upload(h->gpy, py, h->stream));
    CK(upload(h->gph64, g64, h->stream));
    CK(upload(h->gph32, g32, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return IOBM_OK;
}

int iobm_set_wait_limit(iobm_handle* h, long long cycles, int inject_stall) {
    if (!h) return IOBM_E_ARG;
    if (cycles < 0 || (inject_stall != 0 && inject_stall != 1))
        return fail(h, IOBM_E_ARG, "wait limit must be >= 0 and inject_stall 0 or 1");
    h->wait_cycles = cycles;
    h->wait_inject = inject_stall;
    return IOBM_OK;
}

int iobm_profile(iobm_handle* h, int enable) {
    if (!h) return IOBM_E_ARG;
    if (enable < 0 || enable > 4) return IOBM_E_ARG;
    h->profile = enable;
    h->prof_ms = 0.0;
    h->prof_launches = 0;
    return IOBM_OK;
}

int iobm_kernel_stats(const iobm_handle* h, double* kernel_ms, long long* kernel_launches) {
    if (!h) return IOBM_E_ARG;
    if (kernel_ms) *kernel_ms = h->prof_ms;
    if (kernel_launches) *kernel_launches = h->prof_launches;
    return IOBM_OK;
}

int iobm_last_solve_stats(const iobm_handle* h, double* ms, long long* launches,
                          long long* iterations_total) {
    if (!h) return IOBM_E_ARG;
    if (ms) *ms = h->last_ms;
    if (launches) *launches = h->last_launches;
    if (iterations_total) *iterations_total = h->last_iters;
    return IOBM_OK;
}

}  // extern "C"
