// Complex 3D finite-difference stencil (Eq. 1 kinetic term + local potential,
// Eqs. 2-4) and the truncated-Laplacian-Green preconditioner (Eq. 10), as one
// z-marching kernel template.
//
// Each CTA owns a TX x TY lateral tile of one RHS and a chunk of z-planes.  It
// marches through its planes keeping the 2*NF+1 z-neighbours of its own
// points in a register queue (the z taps cost no memory traffic) and stages
// the current plane, with an NF-point periodic halo in x and y, in shared
// memory for the lateral taps.  Planes beyond 0 and nz-1 are zero (Eq. 4:
// the truncated operator; the self-energy kernel adds the boundary term).
//
// In FP32 the taps are applied in difference form, c_n (x_{+n} + x_{-n} - 2 x_0):
// for the kinetic operator the weights sum to zero, so the large diagonal
// cancels analytically and the FP32 result keeps the precision of the smooth
// components (the centre coefficient c0 passed in is the diagonal plus
// 2 sum_n c_n, which is zero for the FD Laplacian).  FP64 has the digits to
// spare and applies the direct form, one FP64 operation fewer per tap pair.
//
// In the fused COCG mode the operand is p = z + beta * p_old, formed on the
// fly wherever p is read and stored once per point by its owning CTA; the
// epilogue accumulates the unconjugated product p^T (A p) (FP32 per thread
// over its planes, FP64 across the CTA) into a per-CTA slot.
#include "iobm_internal.cuh"
#include "complex_ops.cuh"
#include "bulk_copy.cuh"

namespace iobm {

constexpr int kTX = 32;
constexpr int kTY = 8;

// One lateral tap pair at a lateral Bloch vector (gauge exp(-i kappa.r)):
// acc + c (x_m + x_p) + i s (x_p - x_m), with c = c_n cos(n theta) and s the signed
// c_n sin(n theta): the taps c_n exp(-+ i n theta) on x_{-+n}.
template <typename C, typename T>
__device__ __forceinline__ C bloch_taps(C acc, C xm, C xp, T c, T s) {
    acc = caxpy(c, cadd(xm, xp), acc);
    const C d = csub(xp, xm);
    acc.x -= s * d.y;
    acc.y += s * d.x;
    return acc;
}

template <typename T, int NF>
__global__ void __launch_bounds__(kTX* kTY) k_stencil(const StencilArgs<T> a) {
    using C = typename Cplx<T>::type;
    constexpr int W = kTX + 2 * NF;
    constexpr int H = kTY + 2 * NF;
    __shared__ C tile[H][W];
    __shared__ double red[3 * (kTX * kTY / 32)];

    const int rhs = blockIdx.z;
    int st = ST_ACTIVE;
    C beta = czero<C>();
    bool first_dir = false;   // first direction: p = z, p_old is not read
    if (a.state) {
        st = a.state[rhs].status;
        if (a.fused_p && !a.state[rhs].first) beta = from_d2<C>(a.state[rhs].beta);
        else if (a.fused_p) first_dir = true;
    }
    if (!((1 << st) & a.mask)) return;

    const int tile_id = blockIdx.x;
    const int tx0 = (tile_id % a.tiles_x) * kTX;
    const int ty0 = (tile_id / a.tiles_x) * kTY;
    const int k0 = blockIdx.y * a.zchunk;
    const int k1 = min(k0 + a.zchunk, a.nz);
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int tid = ly * kTX + lx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int gx = tx0 + lx, gy = ty0 + ly;
    const bool own = (gx < nx) && (gy < ny);
    const long long plane = (long long)nx * ny;
    const long long base = (long long)rhs * a.npts;
    const C* __restrict__ X = a.x + base;
    const int pb = (a.fused_p && a.state) ? (a.state[rhs].pbuf & 1) : 0;
    const C* __restrict__ PO = (a.fused_p && !first_dir) ? a.pbufs[pb] + base : nullptr;
    C* __restrict__ Y = a.y + base;
    C* __restrict__ PN = a.fused_p ? a.pbufs[1 - pb] + base : nullptr;
    const T ed = a.ediag ? (T)a.ediag[a.rhs_energy ? a.rhs_energy[rhs] : 0] : (T)0;
    const T cen = a.c0 + ed;
    const int sg = (sizeof(T) == 8 && a.rhs_sign) ? a.rhs_sign[rhs] : 0;   // Bloch phase sign
    T tapsum2 = 0;   // 2 sum_n (c_x,n + c_y,n + c_z,n): moves the taps' diagonal into the direct form
#pragma unroll
    for (int n = 1; n <= NF; ++n) tapsum2 += 2 * (a.cx[n] + a.cy[n] + a.cz[n]);

    auto ld = [&](int k, long long lat) -> C {
        if (k < 0 || k >= nz) return czero<C>();
        const long long i = (long long)k * plane + lat;
        C v = X[i];
        if (PO) v = cfma(beta, PO[i], v);
        return v;
    };

    const long long own_lat = own ? (long long)gy * nx + gx : 0;
    C q[2 * NF + 1];
#pragma unroll
    for (int j = 0; j < 2 * NF; ++j) {
        const int kk = k0 - NF + j;
        q[j] = own ? ld(kk, own_lat) : czero<C>();
        if (PN && own && kk >= k0 && kk < k1) PN[(long long)kk * plane + own_lat] = q[j];
    }

    float dre = 0.f, dim = 0.f, nrm = 0.f;   // per-thread partials (FP32 over own planes)
    double dre64 = 0.0, dim64 = 0.0, nrm64 = 0.0;

    for (int k = k0; k < k1; ++k) {
        // own value of plane k+NF enters the queue
        {
            const int kk = k + NF;
            q[2 * NF] = own ? ld(kk, own_lat) : czero<C>();
            if (PN && own && kk < k1) PN[(long long)kk * plane + own_lat] = q[2 * NF];
        }
        __syncthreads();   // previous plane's lateral taps are done
        for (int i = tid; i < W * H; i += kTX * kTY) {
            const int sx = i % W, sy = i / W;
            int ix = tx0 + sx - NF, iy = ty0 + sy - NF;
            ix %= nx; if (ix < 0) ix += nx;
            iy %= ny; if (iy < 0) iy += ny;
            tile[sy][sx] = ld(k, (long long)iy * nx + ix);
        }
        __syncthreads();
        if (own) {
            T d = cen;
            if (a.V) d += a.vsign * a.V[(long long)k * plane + own_lat];
            const C x0 = q[NF];
            C acc;
            if constexpr (sizeof(T) == 8) {
                // FP64: direct form, the diagonal carries -2 sum c_n
                acc = cscale(x0, d - tapsum2);
                if (sg == 0) {
#pragma unroll
                    for (int n = 1; n <= NF; ++n) {
                        acc = caxpy(a.cz[n], cadd(q[NF - n], q[NF + n]), acc);
                        acc = caxpy(a.cx[n], cadd(tile[ly + NF][lx + NF - n], tile[ly + NF][lx + NF + n]), acc);
                        acc = caxpy(a.cy[n], cadd(tile[ly + NF - n][lx + NF], tile[ly + NF + n][lx + NF]), acc);
                    }
                } else {
#pragma unroll
                    for (int n = 1; n <= NF; ++n) {
                        acc = caxpy(a.cz[n], cadd(q[NF - n], q[NF + n]), acc);
                        acc = bloch_taps(acc, tile[ly + NF][lx + NF - n], tile[ly + NF][lx + NF + n],
                                         a.bxc[n], sg * a.bxs[n]);
                        acc = bloch_taps(acc, tile[ly + NF - n][lx + NF], tile[ly + NF + n][lx + NF],
                                         a.byc[n], sg * a.bys[n]);
                    }
                }
            } else {
                const C x2 = cadd(x0, x0);
                acc = cscale(x0, d);
#pragma unroll
                for (int n = 1; n <= NF; ++n) {
                    // difference form: c_n (x_{+n} + x_{-n} - 2 x_0), the kinetic diagonal cancels
                    acc = caxpy(a.cz[n], csub(cadd(q[NF - n], q[NF + n]), x2), acc);
                    acc = caxpy(a.cx[n], csub(cadd(tile[ly + NF][lx + NF - n], tile[ly + NF][lx + NF + n]), x2), acc);
                    acc = caxpy(a.cy[n], csub(cadd(tile[ly + NF - n][lx + NF], tile[ly + NF + n][lx + NF]), x2), acc);
                }
            }
            Y[(long long)k * plane + own_lat] = acc;
            if (a.dot_mode) {
                const C p = q[NF];
                if constexpr (sizeof(T) == 4) {
                    dre = fmaf((float)p.x, (float)acc.x, fmaf(-(float)p.y, (float)acc.y, dre));
                    dim = fmaf((float)p.x, (float)acc.y, fmaf((float)p.y, (float)acc.x, dim));
                    nrm = fmaf((float)p.x, (float)p.x, fmaf((float)p.y, (float)p.y, nrm));
                } else {
                    dre64 += (double)p.x * acc.x - (double)p.y * acc.y;
                    dim64 += (double)p.x * acc.y + (double)p.y * acc.x;
                    nrm64 += (double)p.x * p.x + (double)p.y * p.y;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 2 * NF; ++j) q[j] = q[j + 1];
    }

    if (a.dot_mode) {
        double r0 = dre64 + (double)dre, r1 = dim64 + (double)dim, r2 = nrm64 + (double)nrm;
        block_reduce_3(r0, r1, r2, red);
        if (tid == 0) {
            const int slot = a.slot_base + blockIdx.x + blockIdx.y * gridDim.x;
            a.dot_part[(long long)rhs * a.slot_stride + slot] = make_double2(r0, r1);
            if (a.nrm_part) a.nrm_part[(long long)rhs * a.slot_stride + slot] = r2;
        }
    }
}

// ---------------------------------------------------------------------------
// Full-row variant for lateral planes with N_f <= nx <= 64: a CTA owns whole
// rows (all nx points of kRowTY consecutive y rows), so the x taps wrap inside
// the shared-memory row and only the y halo (N_f rows above and below,
// periodic) is fetched per plane; the CTA's own rows are written into shared
// memory from the register z-queue.  Per point and plane this reads the own
// value of plane k+N_f once and about 2 N_f / kRowTY halo values.
constexpr int kRowTY = 8;

template <typename T>
cudaError_t launch_stencil_tiles(const StencilArgs<T>& a0, int nrhs, cudaStream_t s);

template <typename T, int NF>
__global__ void __launch_bounds__(512) k_stencil_rows(const StencilArgs<T> a) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);             // [kRowTY + 2 NF][nx]
    __shared__ double red[3 * 16];

    const int rhs = blockIdx.z;
    int st = ST_ACTIVE;
    C beta = czero<C>();
    bool first_dir = false;
    if (a.state) {
        st = a.state[rhs].status;
        if (a.fused_p && !a.state[rhs].first) beta = from_d2<C>(a.state[rhs].beta);
        else if (a.fused_p) first_dir = true;
    }
    if (!((1 << st) & a.mask)) return;

    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int tid = threadIdx.x;
    const int x = tid % nx;
    const int ly = tid / nx;                 // 0 .. kRowTY-1
    const int ty0 = blockIdx.x * kRowTY;
    const int rows = min(kRowTY, ny - ty0);  // own rows of this tile
    const bool own = ly < rows;
    const int k0 = blockIdx.y * a.zchunk;
    const int k1 = min(k0 + a.zchunk, nz);
    const long long plane = (long long)nx * ny;
    const long long base = (long long)rhs * a.npts;
    const C* __restrict__ X = a.x + base;
    const int pb = (a.fused_p && a.state) ? (a.state[rhs].pbuf & 1) : 0;
    const C* __restrict__ PO = (a.fused_p && !first_dir) ? a.pbufs[pb] + base : nullptr;
    C* __restrict__ Y = a.y + base;
    C* __restrict__ PN = a.fused_p ? a.pbufs[1 - pb] + base : nullptr;
    const T ed = a.ediag ? (T)a.ediag[a.rhs_energy ? a.rhs_energy[rhs] : 0] : (T)0;
    const T cen = a.c0 + ed;
    const int sg = (sizeof(T) == 8 && a.rhs_sign) ? a.rhs_sign[rhs] : 0;   // Bloch phase sign
    T tapsum2 = 0;   // 2 sum_n (c_x,n + c_y,n + c_z,n): moves the taps' diagonal into the direct form
#pragma unroll
    for (int n = 1; n <= NF; ++n) tapsum2 += 2 * (a.cx[n] + a.cy[n] + a.cz[n]);

    auto ld = [&](int k, long long lat) -> C {
        if (k < 0 || k >= nz) return czero<C>();
        const long long i = (long long)k * plane + lat;
        C v = X[i];
        if (PO) v = cfma(beta, PO[i], v);
        return v;
    };

    // shared-memory rows this thread fetches every plane (halo rows and the rows
    // of a partial tile): s = ly and s = ly + kRowTY, skipping own rows
    constexpr int SR = kRowTY + 2 * NF;
    // the (at most two) shared-memory rows this thread fills from global memory
    bool hf[2];
    int hsm[2];
    long long hlat[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int srow = ly + t * kRowTY;
        hf[t] = srow < SR && !(srow >= NF && srow < NF + rows);
        int gy = ty0 - NF + srow;
        gy %= ny;
        if (gy < 0) gy += ny;
        hsm[t] = srow * nx + x;
        hlat[t] = (long long)gy * nx + x;
    }
    const long long own_lat = own ? (long long)(ty0 + ly) * nx + x : 0;

    C q[2 * NF + 1];
#pragma unroll
    for (int j = 0; j < 2 * NF; ++j) {
        const int kk = k0 - NF + j;
        q[j] = own ? ld(kk, own_lat) : czero<C>();
        if (PN && own && kk >= k0 && kk < k1) PN[(long long)kk * plane + own_lat] = q[j];
    }

    float dre = 0.f, dim = 0.f, nrm = 0.f;
    double dre64 = 0.0, dim64 = 0.0, nrm64 = 0.0;
    C* row = tile + (NF + ly) * nx;

    // Software pipeline: the raw operands (z and p_old) of the own value of
    // plane k+1+NF and of the halo of plane k+1 are loaded during plane k and
    // only combined (p = z + beta p_old) when plane k+1 is processed, so no
    // load is waited on in the iteration that issues it.
    auto raw = [&](int k, long long lat, C& zv, C& pv) {
        if (k < 0 || k >= nz) {
            zv = czero<C>();
            pv = czero<C>();
            return;
        }
        const long long i = (long long)k * plane + lat;
        zv = X[i];
        pv = PO ? PO[i] : czero<C>();
    };
    C oz, op;                 // own, plane k+NF
    C hz[2], hp[2];           // halo, plane k
    raw(own ? k0 + NF : -1, own_lat, oz, op);
#pragma unroll
    for (int t = 0; t < 2; ++t) raw(hf[t] ? k0 : -1, hlat[t], hz[t], hp[t]);

    for (int k = k0; k < k1; ++k) {
        // combine the operands that arrived during the previous plane
        q[2 * NF] = cfma(beta, op, oz);
        if (PN && own && k + NF < k1) PN[(long long)(k + NF) * plane + own_lat] = q[2 * NF];
        C hv[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) hv[t] = cfma(beta, hp[t], hz[t]);
        // issue the loads for the next plane
        raw(own ? k + 1 + NF : -1, own_lat, oz, op);
#pragma unroll
        for (int t = 0; t < 2; ++t) raw((hf[t] && k + 1 < k1) ? k + 1 : -1, hlat[t], hz[t], hp[t]);
        __syncthreads();   // previous plane's taps are done
#pragma unroll
        for (int t = 0; t < 2; ++t)
            if (hf[t]) tile[hsm[t]] = hv[t];
        if (own) row[x] = q[NF];
        __syncthreads();
        if (own) {
            T d = cen;
            if (a.V) d += a.vsign * a.V[(long long)k * plane + own_lat];
            const C x0 = q[NF];
            C acc;
            if constexpr (sizeof(T) == 8) {
                // FP64: direct form, the diagonal carries -2 sum c_n (2 instead of 3
                // FP64 operations per tap pair and component; the FP64 ALU is the limit)
                acc = cscale(x0, d - tapsum2);
                if (sg == 0) {
#pragma unroll
                    for (int n = 1; n <= NF; ++n) {
                        const int xm = (x - n < 0) ? x - n + nx : x - n;
                        const int xp = (x + n >= nx) ? x + n - nx : x + n;
                        acc = caxpy(a.cz[n], cadd(q[NF - n], q[NF + n]), acc);
                        acc = caxpy(a.cx[n], cadd(row[xm], row[xp]), acc);
                        acc = caxpy(a.cy[n], cadd(row[x - n * nx], row[x + n * nx]), acc);
                    }
                } else {
#pragma unroll
                    for (int n = 1; n <= NF; ++n) {
                        const int xm = (x - n < 0) ? x - n + nx : x - n;
                        const int xp = (x + n >= nx) ? x + n - nx : x + n;
                        acc = caxpy(a.cz[n], cadd(q[NF - n], q[NF + n]), acc);
                        acc = bloch_taps(acc, row[xm], row[xp], a.bxc[n], sg * a.bxs[n]);
                        acc = bloch_taps(acc, row[x - n * nx], row[x + n * nx], a.byc[n], sg * a.bys[n]);
                    }
                }
            } else {
                const C x2 = cadd(x0, x0);
                acc = cscale(x0, d);
#pragma unroll
                for (int n = 1; n <= NF; ++n) {
                    const int xm = (x - n < 0) ? x - n + nx : x - n;     // periodic in x (nx >= NF)
                    const int xp = (x + n >= nx) ? x + n - nx : x + n;
                    acc = caxpy(a.cz[n], csub(cadd(q[NF - n], q[NF + n]), x2), acc);
                    acc = caxpy(a.cx[n], csub(cadd(row[xm], row[xp]), x2), acc);
                    acc = caxpy(a.cy[n], csub(cadd(row[x - n * nx], row[x + n * nx]), x2), acc);
                }
            }
            Y[(long long)k * plane + own_lat] = acc;
            if (a.dot_mode) {
                const C p = x0;
                if constexpr (sizeof(T) == 4) {
                    dre = fmaf((float)p.x, (float)acc.x, fmaf(-(float)p.y, (float)acc.y, dre));
                    dim = fmaf((float)p.x, (float)acc.y, fmaf((float)p.y, (float)acc.x, dim));
                    nrm = fmaf((float)p.x, (float)p.x, fmaf((float)p.y, (float)p.y, nrm));
                } else {
                    dre64 += (double)p.x * acc.x - (double)p.y * acc.y;
                    dim64 += (double)p.x * acc.y + (double)p.y * acc.x;
                    nrm64 += (double)p.x * p.x + (double)p.y * p.y;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 2 * NF; ++j) q[j] = q[j + 1];
    }

    if (a.dot_mode) {
        double r0 = dre64 + (double)dre, r1 = dim64 + (double)dim, r2 = nrm64 + (double)nrm;
        block_reduce_3(r0, r1, r2, red);
        if (tid == 0) {
            const int slot = a.slot_base + blockIdx.x + blockIdx.y * gridDim.x;
            a.dot_part[(long long)rhs * a.slot_stride + slot] = make_double2(r0, r1);
            if (a.nrm_part) a.nrm_part[(long long)rhs * a.slot_stride + slot] = r2;
        }
    }
}

// ---------------------------------------------------------------------------
// Full-row variant with the operands staged by bulk copies (FP32, row widths
// NX of the compile-time FFT plans).  Same tiling and arithmetic as
// k_stencil_rows, but the raw operands (z and p_old) of every plane arrive in
// shared memory through cp.async.bulk copies issued kTmaStages planes ahead
// into a ring of stages, each completing on its own mbarrier; no thread waits
// on a global load.  Stage s holds, for plane k, the own rows of plane k+N_f
// (they enter the register z-queue) and the N_f halo rows above and below of
// plane k (they go to the row tile): one contiguous copy for the own rows and
// one per halo row (the periodic wrap in y is a matter of the source row
// index), issued by the lanes of warp 0 in parallel.  The row tile carries N_f
// periodic pad columns on each side, so every tap is a constant offset, and is
// double-buffered: one CTA barrier per plane separates the stage reads and
// tile writes of plane k from the copies into the freed stage and the taps of
// plane k.
constexpr int kTmaStages = 4;

template <int NX, int NF>
struct RowsTma {
    static constexpr int SR = kRowTY + 2 * NF;   // tile / stage rows
    static constexpr int TP = NX + 2 * NF;       // tile pitch (periodic pad columns)
    static constexpr int TILE = SR * TP;
    static constexpr int SLAB = SR * NX;
    static constexpr size_t smem = 128 + sizeof(float2) * (2 * (size_t)TILE + 2 * (size_t)kTmaStages * SLAB);
};

template <int NX, int NF, int MINB>
__global__ void __launch_bounds__(NX * kRowTY, MINB) k_stencil_rows_tma(const StencilArgs<float> a) {
    using T = float;
    using C = float2;
    using L = RowsTma<NX, NF>;
    constexpr int TP = L::TP, TILE = L::TILE, SLAB = L::SLAB;
    constexpr int D = kTmaStages;
    extern __shared__ __align__(128) unsigned char smem_tma[];
    __shared__ double red[3 * 16];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_tma);   // [D]

    const int rhs = blockIdx.z;
    int st = ST_ACTIVE;
    C beta = czero<C>();
    bool first_dir = false;
    if (a.state) {
        st = a.state[rhs].status;
        if (a.fused_p && !a.state[rhs].first) beta = from_d2<C>(a.state[rhs].beta);
        else if (a.fused_p) first_dir = true;
    }
    if (!((1 << st) & a.mask)) return;

    const int ny = a.ny, nz = a.nz;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int x = tid % NX;
    const int ly = tid / NX;
    const int ty0 = blockIdx.x * kRowTY;
    const int rows = min(kRowTY, ny - ty0);
    const bool own = ly < rows;
    const int k0 = blockIdx.y * a.zchunk;
    const int k1 = min(k0 + a.zchunk, nz);
    const long long plane = (long long)NX * ny;
    const long long base = (long long)rhs * a.npts;
    const C* __restrict__ X = a.x + base;
    const int pb = (a.fused_p && a.state) ? (a.state[rhs].pbuf & 1) : 0;
    const C* __restrict__ PO = (a.fused_p && !first_dir) ? a.pbufs[pb] + base : nullptr;
    const T ed = a.ediag ? (T)a.ediag[a.rhs_energy ? a.rhs_energy[rhs] : 0] : (T)0;
    const T cen = a.c0 + ed;

    C* tiles = reinterpret_cast<C*>(smem_tma + 128);   // [2][SR][TP] combined operand rows
    C* stages = tiles + 2 * TILE;                      // stage s: z at 2 s SLAB, p_old at (2 s + 1) SLAB
    if (tid == 0) {
        for (int s = 0; s <= D; ++s) mbar_init(&bar[s], 1);   // bar[D]: no copy completes it
        mbar_init_fence();
    }
    __syncthreads();
    const long long wlim = a.wait_cycles > 0 ? a.wait_cycles : kWaitCycles;

    // copy assignment of warp 0.  A halo side (NF rows above or below the own
    // rows) whose source rows do not wrap around in y is one copy of NF rows,
    // otherwise one copy per row.  Lane l < 2 NF: halo row l (row copies of a
    // wrapping side; for a contiguous side its first lane copies all NF rows);
    // lane 2 NF: the own rows of z, lane 2 NF + 1: those of p_old.
    constexpr uint32_t row_bytes = NX * sizeof(C);
    auto issue = [&](int k, int s) {   // all lanes of warp 0
        const bool own_plane = k + NF < nz;
        if (lane == 0) {
            const uint32_t per = (own_plane ? (uint32_t)rows : 0u) * row_bytes + 2u * NF * row_bytes;
            mbar_arrive_expect_tx(&bar[s], PO ? 2 * per : per);
        }
        __syncwarp();
        C* sz = stages + 2 * s * SLAB;
        C* sp = sz + SLAB;
        if (lane < 2 * NF) {
            const bool above = lane < NF;
            const int h = above ? lane : lane - NF;
            const bool contiguous = above ? (ty0 >= NF) : (ty0 + rows + NF <= ny);
            const int nrows = contiguous ? (h == 0 ? NF : 0) : 1;
            if (nrows) {
                const int srow = above ? lane : NF + rows + h;
                int gy = (ty0 - NF + srow) % ny;
                if (gy < 0) gy += ny;
                fence_proxy_async_smem();
                const long long src = (long long)k * plane + (long long)gy * NX;
                bulk_g2s(sz + srow * NX, X + src, nrows * row_bytes, &bar[s]);
                if (PO) bulk_g2s(sp + srow * NX, PO + src, nrows * row_bytes, &bar[s]);
            }
        } else if (own_plane && (lane == 2 * NF || (PO && lane == 2 * NF + 1))) {
            fence_proxy_async_smem();
            const long long src = (long long)(k + NF) * plane + (long long)ty0 * NX;
            if (lane == 2 * NF) bulk_g2s(sz + NF * NX, X + src, rows * row_bytes, &bar[s]);
            else bulk_g2s(sp + NF * NX, PO + src, rows * row_bytes, &bar[s]);
        }
    };

    // tile rows this thread fills from the stage (the halo rows of a full or
    // partial tile): stage rows ly and ly + kRowTY, stage index tid + t kRowTY NX
    bool hf[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int srow = ly + t * kRowTY;
        hf[t] = srow < 2 * NF + rows && !(srow >= NF && srow < NF + rows);
    }
    // column of x in the padded tile, and its periodic copy in the pad (or -1;
    // NX >= 2 NF, so a column has at most one copy)
    static_assert(NX >= 2 * NF, "pad columns assume NX >= 2 NF");
    const int tcol = NF + x;
    const int tpad = (x < NF) ? NF + NX + x : ((x >= NX - NF) ? x - (NX - NF) : -1);
    const long long own_lat = own ? (long long)(ty0 + ly) * NX + x : 0;

    auto ld = [&](int k, long long lat) -> C {
        if (k < 0 || k >= nz) return czero<C>();
        const long long i = (long long)k * plane + lat;
        C v = X[i];
        if (PO) v = cfma(beta, PO[i], v);
        return v;
    };
    if (tid < 32)
        for (int j = 0; j < D && k0 + j < k1; ++j) issue(k0 + j, j);

    C* PN = a.fused_p ? a.pbufs[1 - pb] + base : nullptr;
    C q[2 * NF + 1];
#pragma unroll
    for (int j = 0; j < 2 * NF; ++j) {
        const int kk = k0 - NF + j;
        q[j] = own ? ld(kk, own_lat) : czero<C>();
        if (PN && own && kk >= k0 && kk < k1) PN[(long long)kk * plane + own_lat] = q[j];
    }
    // running pointers at plane k (Y, V) and k + NF (PN)
    C* __restrict__ Yk = a.y + base + (long long)k0 * plane + own_lat;
    C* __restrict__ PNk = PN ? PN + (long long)(k0 + NF) * plane + own_lat : nullptr;
    const T* __restrict__ Vk = a.V ? a.V + (long long)k0 * plane + own_lat : nullptr;
    T vnext = (Vk && own) ? Vk[0] : (T)0;

    float dre = 0.f, dim = 0.f, nrm = 0.f;
    const int own_st = (NF + ly) * NX + x;

    for (int k = k0; k < k1; ++k) {
        const unsigned kk = (unsigned)(k - k0);
        const int s = (int)(kk % D);
        C* tile = tiles + (kk & 1) * TILE;
        const T vk = vnext;
        if (Vk && own && k + 1 < k1) vnext = Vk[plane];
        bool ok = mbar_wait_bounded(&bar[s], (kk / D) & 1, wlim);
        if (a.wait_inject && kk == 0 && tid == 0) ok = ok && mbar_wait_bounded(&bar[D], 0, wlim);
        const C* sz = stages + 2 * s * SLAB;
        const C* sp = sz + SLAB;
        C qn = czero<C>();
        if (own && k + NF < nz) {
            const C zv = sz[own_st];
            qn = PO ? cfma(beta, sp[own_st], zv) : zv;
        }
        q[2 * NF] = qn;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (hf[t]) {
                const int si = tid + t * kRowTY * NX;
                const C zv = sz[si];
                const C v = PO ? cfma(beta, sp[si], zv) : zv;
                C* trow = tile + (ly + t * kRowTY) * TP;
                trow[tcol] = v;
                if (tpad >= 0) trow[tpad] = v;
            }
        }
        C* row = tile + (NF + ly) * TP;
        if (own) {
            row[tcol] = q[NF];
            if (tpad >= 0) row[tpad] = q[NF];
        }
        // stage s is consumed and tile k is complete; the other tile (plane k-1)
        // was last read before this barrier
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                if (a.err) atomicExch(a.err, ERR_STAGE_TIMEOUT);
                for (int j = k; j < k + D && j < k1; ++j)   // this CTA's copies still in flight
                    mbar_wait_bounded(&bar[(j - k0) % D], ((j - k0) / D) & 1);
            }
            __syncthreads();
            return;
        }
        if (tid < 32 && k + D < k1) issue(k + D, s);
        if (PNk && own && k + NF < k1) PNk[0] = qn;
        if (own) {
            T d = cen;
            if (Vk) d += a.vsign * vk;
            const C x0 = q[NF];
            const C* c = row + tcol;
            C acc;
            if (a.iso) {
                // the same difference form in packed two-lane FP32 instructions (one
                // weight pair per shift n serves all three axes)
                const C x2 = p2add(x0, x0);
                acc = p2mul(x0, make_float2(d, d));
#pragma unroll
                for (int n = 1; n <= NF; ++n) {
                    const C cc = make_float2(a.cz[n], a.cz[n]);
                    acc = p2fma(cc, p2sub(p2add(q[NF - n], q[NF + n]), x2), acc);
                    acc = p2fma(cc, p2sub(p2add(c[-n], c[n]), x2), acc);
                    acc = p2fma(cc, p2sub(p2add(c[-n * TP], c[n * TP]), x2), acc);
                }
            } else {
                const C x2 = cadd(x0, x0);
                acc = cscale(x0, d);
#pragma unroll
                for (int n = 1; n <= NF; ++n) {
                    acc = caxpy(a.cz[n], csub(cadd(q[NF - n], q[NF + n]), x2), acc);
                    acc = caxpy(a.cx[n], csub(cadd(c[-n], c[n]), x2), acc);
                    acc = caxpy(a.cy[n], csub(cadd(c[-n * TP], c[n * TP]), x2), acc);
                }
            }
            Yk[0] = acc;
            if (a.dot_mode) {
                dre = fmaf(x0.x, acc.x, fmaf(-x0.y, acc.y, dre));
                dim = fmaf(x0.x, acc.y, fmaf(x0.y, acc.x, dim));
                nrm = fmaf(x0.x, x0.x, fmaf(x0.y, x0.y, nrm));
            }
        }
        Yk += plane;
        if (PNk) PNk += plane;
        if (Vk) Vk += plane;
#pragma unroll
        for (int j = 0; j < 2 * NF; ++j) q[j] = q[j + 1];
    }

    if (a.dot_mode) {
        double r0 = dre, r1 = dim, r2 = nrm;
        block_reduce_3(r0, r1, r2, red);
        if (tid == 0) {
            const int slot = a.slot_base + blockIdx.x + blockIdx.y * gridDim.x;
            a.dot_part[(long long)rhs * a.slot_stride + slot] = make_double2(r0, r1);
            if (a.nrm_part) a.nrm_part[(long long)rhs * a.slot_stride + slot] = r2;
        }
    }
}

// ---------------------------------------------------------------------------
// Blocked bulk-copy variant (FP32, row widths of the compile-time FFT plans, ny a
// multiple of RY): the staging, tile and arithmetic of k_stencil_rows_tma, but each
// thread owns PT consecutive rows of one x column, so a CTA of NX x TY threads covers
// RY = TY PT rows.  The per-plane work of a thread (stage wait, CTA barrier, loop and
// address arithmetic, its share of the halo fill) then serves PT points, and the y
// taps between a thread's own rows come from its registers: per plane a thread reads
// 2 N_f tile values for its y taps instead of 2 N_f per point.  The potential of the
// own rows arrives with the stage (one more bulk copy), and the taps accumulate per
// axis (three independent chains).
template <int NX, int NF, int PT, int TY, int D_ = 3>
struct BlkTma {
    static constexpr int RY = TY * PT;           // own rows of a CTA
    static constexpr int SR = RY + 2 * NF;       // tile / stage rows
    static constexpr int TP = NX + 2 * NF;       // tile pitch (periodic pad columns)
    static constexpr int TILE = SR * TP;
    static constexpr int SLAB = SR * NX;
    static constexpr int VSLAB = RY * NX / 2;    // float2 units holding RY x NX floats
    static constexpr int D = D_;                 // stages (copies issued D planes ahead)
    static constexpr int STAGE = 2 * SLAB + VSLAB;
    static constexpr size_t smem = 128 + sizeof(float2) * (2 * (size_t)TILE + (size_t)D * STAGE);
};

template <int NX, int NF, int PT, int TY, int MINB, int DS>
__global__ void __launch_bounds__(NX * TY, MINB) k_stencil_blk(const StencilArgs<float> a) {
    using T = float;
    using C = float2;
    using L = BlkTma<NX, NF, PT, TY, DS>;
    constexpr int TP = L::TP, TILE = L::TILE, SLAB = L::SLAB, RY = L::RY, D = L::D;
    constexpr int STAGE = L::STAGE;
    extern __shared__ __align__(128) unsigned char smem_blk[];
    __shared__ double red[3 * 16];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_blk);   // [D + 1]

    const int rhs = blockIdx.z;
    int st = ST_ACTIVE;
    C beta = czero<C>();
    bool first_dir = false;
    if (a.state) {
        st = a.state[rhs].status;
        if (a.fused_p && !a.state[rhs].first) beta = from_d2<C>(a.state[rhs].beta);
        else if (a.fused_p) first_dir = true;
    }
    if (!((1 << st) & a.mask)) return;

    const int ny = a.ny, nz = a.nz;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int x = tid % NX;
    const int ty = tid / NX;                 // 0 .. TY-1
    const int r0 = ty * PT;                  // this thread's first own row within the tile
    const int ty0 = blockIdx.x * RY;         // first own row of the tile (full tiles only)
    const int k0 = blockIdx.y * a.zchunk;
    const int k1 = min(k0 + a.zchunk, nz);
    const long long plane = (long long)NX * ny;
    const long long base = (long long)rhs * a.npts;
    const C* __restrict__ X = a.x + base;
    const int pb = (a.fused_p && a.state) ? (a.state[rhs].pbuf & 1) : 0;
    const C* __restrict__ PO = (a.fused_p && !first_dir) ? a.pbufs[pb] + base : nullptr;
    const T* __restrict__ Vg = a.V;
    const T ed = a.ediag ? (T)a.ediag[a.rhs_energy ? a.rhs_energy[rhs] : 0] : (T)0;
    const T cen = a.c0 + ed;

    C* tiles = reinterpret_cast<C*>(smem_blk + 128);   // [2][SR][TP] combined operand rows
    C* stages = tiles + 2 * TILE;   // stage s at s STAGE: z [SLAB], p_old [SLAB], V [RY][NX] floats
    if (tid == 0) {
        for (int s = 0; s <= D; ++s) mbar_init(&bar[s], 1);   // bar[D]: no copy completes it
        mbar_init_fence();
    }
    __syncthreads();
    const long long wlim = a.wait_cycles > 0 ? a.wait_cycles : kWaitCycles;

    // copies of warp 0 (as in k_stencil_rows_tma, with RY own rows): lane l < 2 NF a
    // halo row (a side whose source rows do not wrap in y is one copy by its first
    // lane), lane 2 NF the own rows of z, lane 2 NF + 1 those of p_old, lane 2 NF + 2
    // the own rows of V (of plane k itself)
    constexpr uint32_t row_bytes = NX * sizeof(C);
    constexpr uint32_t vrow_bytes = NX * sizeof(T);
    auto issue = [&](int k, int s) {   // all lanes of warp 0
        const bool own_plane = k + NF < nz;
        if (lane == 0) {
            const uint32_t per = (own_plane ? (uint32_t)RY : 0u) * row_bytes + 2u * NF * row_bytes;
            mbar_arrive_expect_tx(&bar[s], (PO ? 2 * per : per) + (Vg ? RY * vrow_bytes : 0u));
        }
        __syncwarp();
        C* sz = stages + s * STAGE;
        C* sp = sz + SLAB;
        if (lane < 2 * NF) {
            const bool above = lane < NF;
            const int h = above ? lane : lane - NF;
            const bool contiguous = above ? (ty0 >= NF) : (ty0 + RY + NF <= ny);
            const int nrows = contiguous ? (h == 0 ? NF : 0) : 1;
            if (nrows) {
                const int srow = above ? lane : NF + RY + h;
                int gy = (ty0 - NF + srow) % ny;
                if (gy < 0) gy += ny;
                fence_proxy_async_smem();
                const long long src = (long long)k * plane + (long long)gy * NX;
                bulk_g2s(sz + srow * NX, X + src, nrows * row_bytes, &bar[s]);
                if (PO) bulk_g2s(sp + srow * NX, PO + src, nrows * row_bytes, &bar[s]);
            }
        } else if (own_plane && (lane == 2 * NF || (PO && lane == 2 * NF + 1))) {
            fence_proxy_async_smem();
            const long long src = (long long)(k + NF) * plane + (long long)ty0 * NX;
            if (lane == 2 * NF) bulk_g2s(sz + NF * NX, X + src, RY * row_bytes, &bar[s]);
            else bulk_g2s(sp + NF * NX, PO + src, RY * row_bytes, &bar[s]);
        } else if (Vg && lane == 2 * NF + 2) {
            fence_proxy_async_smem();
            bulk_g2s(sz + 2 * SLAB, Vg + (long long)k * plane + (long long)ty0 * NX, RY * vrow_bytes,
                     &bar[s]);
        }
    };

    static_assert(NX >= 2 * NF, "pad columns assume NX >= 2 NF");
    const int tcol = NF + x;
    const int tpad = (x < NF) ? NF + NX + x : ((x >= NX - NF) ? x - (NX - NF) : -1);
    const long long own_lat = (long long)(ty0 + r0) * NX + x;   // own row i at + i NX

    auto ld = [&](int k, long long lat) -> C {
        if (k < 0 || k >= nz) return czero<C>();
        const long long i = (long long)k * plane + lat;
        C v = X[i];
        if (PO) v = cfma(beta, PO[i], v);
        return v;
    };
    if (tid < 32)
        for (int j = 0; j < D && k0 + j < k1; ++j) issue(k0 + j, j);

    C* PN = a.fused_p ? a.pbufs[1 - pb] + base : nullptr;
    C q[2 * NF + 1][PT];
#pragma unroll
    for (int j = 0; j < 2 * NF; ++j) {
        const int kk = k0 - NF + j;
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            q[j][i] = ld(kk, own_lat + i * NX);
            if (PN && kk >= k0 && kk < k1) PN[(long long)kk * plane + own_lat + i * NX] = q[j][i];
        }
    }
    C* __restrict__ Yk = a.y + base + (long long)k0 * plane + own_lat;
    C* __restrict__ PNk = PN ? PN + (long long)(k0 + NF) * plane + own_lat : nullptr;

    float dre = 0.f, dim = 0.f, nrm = 0.f;
    constexpr int HF = (2 * NF + TY - 1) / TY;   // halo rows filled per thread

    // Software pipeline, one CTA barrier per plane: the barrier interval of plane k
    // computes the outputs of plane k from tile buffer k & 1 while it fills buffer
    // (k + 1) & 1 from the stage of plane k + 1 (its halo rows, the own rows from the
    // z-queue) and takes the own rows of plane k + 1 + NF into the queue.
    T vk[PT], vn[PT];
    C qn[PT];
    // fill of plane kf into tile buffer (kf - k0) & 1: the stage of kf must have arrived
    auto fill = [&](int kf, T* vout) {
        const unsigned kk = (unsigned)(kf - k0);
        const C* sz = stages + (int)(kk % D) * STAGE;
        const C* sp = sz + SLAB;
        const T* sv = reinterpret_cast<const T*>(sz + 2 * SLAB) + r0 * NX + x;
        C* tile = tiles + (kk & 1) * TILE;
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            qn[i] = czero<C>();
            if (kf + NF < nz) {
                const int si = (NF + r0 + i) * NX + x;
                const C zv = sz[si];
                qn[i] = PO ? cfma(beta, sp[si], zv) : zv;
            }
            vout[i] = Vg ? sv[i * NX] : (T)0;
        }
#pragma unroll
        for (int jj = 0; jj < HF; ++jj) {
            const int j = ty + jj * TY;
            if (j < 2 * NF) {
                const int srow = j < NF ? j : RY + j;
                const int si = srow * NX + x;
                const C zv = sz[si];
                const C v = PO ? cfma(beta, sp[si], zv) : zv;
                C* trow = tile + srow * TP;
                trow[tcol] = v;
                if (tpad >= 0) trow[tpad] = v;
            }
        }
    };
    // own rows of plane kf (held in the queue) into its tile buffer
    auto own_rows = [&](int kf, const C* vals) {
        C* tile = tiles + ((unsigned)(kf - k0) & 1) * TILE;
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            C* row = tile + (NF + r0 + i) * TP;
            row[tcol] = vals[i];
            if (tpad >= 0) row[tpad] = vals[i];
        }
    };
    // a CTA barrier that also agrees on a failed wait; on failure the CTA drains the
    // copies it still has in flight (planes kw .. kw + D - 1) and the kernel returns
    auto barrier_ok = [&](bool ok, int kw) -> bool {
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                if (a.err) atomicExch(a.err, ERR_STAGE_TIMEOUT);
                for (int j = kw; j < kw + D && j < k1; ++j)
                    mbar_wait_bounded(&bar[(j - k0) % D], ((j - k0) / D) & 1);
            }
            __syncthreads();
            return false;
        }
        return true;
    };

    // prologue: plane k0 into tile buffer 0
    {
        bool ok = mbar_wait_bounded(&bar[0], 0, wlim);
        if (a.wait_inject && tid == 0) ok = ok && mbar_wait_bounded(&bar[D], 0, wlim);
        fill(k0, vk);
        C own0[PT];
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            own0[i] = q[NF][i];
            q[2 * NF][i] = qn[i];
        }
        own_rows(k0, own0);
        if (!barrier_ok(ok, k0)) return;
        if (tid < 32 && k0 + D < k1) issue(k0 + D, 0);
        if (PNk && k0 + NF < k1) {
#pragma unroll
            for (int i = 0; i < PT; ++i) PNk[i * NX] = qn[i];
        }
        if (PNk) PNk += plane;
    }

    for (int k = k0; k < k1; ++k) {
        const unsigned kk = (unsigned)(k - k0);
        const C* tile = tiles + (kk & 1) * TILE;
        const bool next = k + 1 < k1;
        bool ok = true;
        if (next) {   // plane k + 1: its stage, tile buffer and queue entry
            ok = mbar_wait_bounded(&bar[(kk + 1) % D], ((kk + 1) / D) & 1, wlim);
            fill(k + 1, vn);
            C own1[PT];
#pragma unroll
            for (int i = 0; i < PT; ++i) own1[i] = q[NF + 1][i];
            own_rows(k + 1, own1);
        }
        // y neighbours outside this thread's rows: NF above, NF below
        C yh[2 * NF];
#pragma unroll
        for (int m = 0; m < NF; ++m) {
            yh[m] = tile[(r0 + m) * TP + tcol];                  // row r0 - NF + m
            yh[NF + m] = tile[(NF + r0 + PT + m) * TP + tcol];   // row r0 + PT + m
        }
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            const T d = cen + a.vsign * vk[i];
            const C x0 = q[NF][i];
            const C* c = tile + (NF + r0 + i) * TP + tcol;
            C acc;
            if (a.iso) {
                // three independent chains (z, x, y taps), summed at the end
                const C x2 = p2add(x0, x0);
                C az = p2mul(x0, make_float2(d, d));
                C ax = make_float2(0.f, 0.f), ay = ax;
#pragma unroll
                for (int n = 1; n <= NF; ++n) {
                    const int dm = i - n, dp = i + n;   // own-relative rows (compile-time)
                    const C ym = dm >= 0 ? q[NF][dm < PT ? dm : PT - 1] : yh[dm + NF >= 0 ? dm + NF : 0];
                    const C yp = dp < PT ? q[NF][dp] : yh[NF + dp - PT < 2 * NF ? NF + dp - PT : 2 * NF - 1];
                    const C cc = make_float2(a.cz[n], a.cz[n]);
                    az = p2fma(cc, p2sub(p2add(q[NF - n][i], q[NF + n][i]), x2), az);
                    ax = p2fma(cc, p2sub(p2add(c[-n], c[n]), x2), ax);
                    ay = p2fma(cc, p2sub(p2add(ym, yp), x2), ay);
                }
                acc = p2add(az, p2add(ax, ay));
            } else {
                const C x2 = cadd(x0, x0);
                C az = cscale(x0, d);
                C ax = make_float2(0.f, 0.f), ay = ax;
#pragma unroll
                for (int n = 1; n <= NF; ++n) {
                    const int dm = i - n, dp = i + n;
                    const C ym = dm >= 0 ? q[NF][dm < PT ? dm : PT - 1] : yh[dm + NF >= 0 ? dm + NF : 0];
                    const C yp = dp < PT ? q[NF][dp] : yh[NF + dp - PT < 2 * NF ? NF + dp - PT : 2 * NF - 1];
                    az = caxpy(a.cz[n], csub(cadd(q[NF - n][i], q[NF + n][i]), x2), az);
                    ax = caxpy(a.cx[n], csub(cadd(c[-n], c[n]), x2), ax);
                    ay = caxpy(a.cy[n], csub(cadd(ym, yp), x2), ay);
                }
                acc = cadd(az, cadd(ax, ay));
            }
            Yk[i * NX] = acc;
            if (a.dot_mode) {
                dre = fmaf(x0.x, acc.x, fmaf(-x0.y, acc.y, dre));
                dim = fmaf(x0.x, acc.y, fmaf(x0.y, acc.x, dim));
                nrm = fmaf(x0.x, x0.x, fmaf(x0.y, x0.y, nrm));
            }
        }
        Yk += plane;
        // tile buffer k & 1 is read, (k + 1) & 1 complete, the stage of plane k + 1 consumed
        if (next) {
            if (!barrier_ok(ok, k + 1)) return;
            if (tid < 32 && k + 1 + D < k1) issue(k + 1 + D, (int)((kk + 1) % D));
            if (PNk && k + 1 + NF < k1) {
#pragma unroll
                for (int i = 0; i < PT; ++i) PNk[i * NX] = qn[i];
            }
            if (PNk) PNk += plane;
        }
#pragma unroll
        for (int j = 0; j < 2 * NF; ++j)
#pragma unroll
            for (int i = 0; i < PT; ++i) q[j][i] = q[j + 1][i];
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            q[2 * NF][i] = qn[i];
            vk[i] = vn[i];
        }
    }

    if (a.dot_mode) {
        // partial slots are numbered per kRowTY-row tile (stencil_slots): the CTA's sum
        // goes to the first of its RY / kRowTY slots, zeros to the others
        static_assert(RY % kRowTY == 0, "RY spans whole row tiles");
        double r0d = dre, r1 = dim, r2 = nrm;
        block_reduce_3(r0d, r1, r2, red);
        if (tid < RY / kRowTY) {
            const int tiles_y = ny / kRowTY;
            const int slot = a.slot_base + blockIdx.x * (RY / kRowTY) + tid + blockIdx.y * tiles_y;
            a.dot_part[(long long)rhs * a.slot_stride + slot] =
                tid == 0 ? make_double2(r0d, r1) : make_double2(0.0, 0.0);
            if (a.nrm_part) a.nrm_part[(long long)rhs * a.slot_stride + slot] = tid == 0 ? r2 : 0.0;
        }
    }
}

// Ring kernel (variant 4): the operand planes k - N_f .. k + N_f of a 16-row tile live
// in a ring of 2 N_f + 2 shared-memory slots (combined p = z + beta p_old, N_f halo rows,
// periodic pad columns), so the z taps come from shared memory like the x and y taps and
// no register z-queue is needed: one thread per tile point (NX x 16 threads), a few
// dozen registers.  Fill step f: wait for the bulk copies of plane f (all tile rows of
// z and p_old, periodic in y), fill its ring slot and write p for the own rows, one CTA
// barrier, issue the copies of plane f + 2, and compute output plane f - N_f from the
// ring.  A slot written at step f + 1 held plane f + 1 - (2 N_f + 2), which only step
// f - 1's outputs read; every thread finished those before the barrier of step f.
template <int NX, int NF>
struct RingTma {
    static constexpr int RY = 16;                // own rows of a CTA
    static constexpr int SR = RY + 2 * NF;       // rows of a slot / stage
    static constexpr int TP = NX + 2 * NF;       // slot pitch (pad columns)
    static constexpr int TILE = SR * TP;
    static constexpr int NR = 2 * NF + 2;        // ring slots
    static constexpr int SLAB = SR * NX;
    static constexpr int D = 2;                  // stages (copies issued D planes ahead)
    static constexpr int STAGE = 2 * SLAB;
    static constexpr int NT = NX * RY;
    static constexpr size_t smem = 128 + sizeof(float2) * ((size_t)NR * TILE + (size_t)D * STAGE);
};

template <int NX, int NF>
__global__ void __launch_bounds__(NX * 16) k_stencil_ring(const StencilArgs<float> a) {
    using T = float;
    using C = float2;
    using L = RingTma<NX, NF>;
    constexpr int RY = L::RY, SR = L::SR, TP = L::TP, TILE = L::TILE, NR = L::NR;
    constexpr int SLAB = L::SLAB, D = L::D, STAGE = L::STAGE, NT = L::NT;
    extern __shared__ __align__(128) unsigned char smem_ring[];
    __shared__ double red[3 * 32];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_ring);   // [D + 1]

    const int rhs = blockIdx.z;
    int st = ST_ACTIVE;
    C beta = czero<C>();
    bool first_dir = false;
    if (a.state) {
        st = a.state[rhs].status;
        if (a.fused_p && !a.state[rhs].first) beta = from_d2<C>(a.state[rhs].beta);
        else if (a.fused_p) first_dir = true;
    }
    if (!((1 << st) & a.mask)) return;

    const int ny = a.ny, nz = a.nz;
    const int tid = threadIdx.x;
    const int x = tid % NX, r = tid / NX;    // own point: row r of the tile's RY rows
    const int ty0 = blockIdx.x * RY;
    const int k0 = blockIdx.y * a.zchunk;
    const int k1 = min(k0 + a.zchunk, nz);
    const long long plane = (long long)NX * ny;
    const long long base = (long long)rhs * a.npts;
    const C* __restrict__ X = a.x + base;
    const int pb = (a.fused_p && a.state) ? (a.state[rhs].pbuf & 1) : 0;
    const C* __restrict__ PO = (a.fused_p && !first_dir) ? a.pbufs[pb] + base : nullptr;
    C* __restrict__ PN = a.fused_p ? a.pbufs[1 - pb] + base : nullptr;
    const T* __restrict__ Vg = a.V;
    const T ed = a.ediag ? (T)a.ediag[a.rhs_energy ? a.rhs_energy[rhs] : 0] : (T)0;
    const T cen = a.c0 + ed;

    C* ring = reinterpret_cast<C*>(smem_ring + 128);   // [NR][SR][TP]
    C* stages = ring + NR * TILE;                        // [D]: z [SLAB], p_old [SLAB]
    if (tid == 0) {
        for (int q = 0; q <= D; ++q) mbar_init(&bar[q], 1);   // bar[D]: no copy completes it
        mbar_init_fence();
    }
    __syncthreads();
    const long long wlim = a.wait_cycles > 0 ? a.wait_cycles : kWaitCycles;

    // copies of plane f into stage q (thread 0): tile rows ty0 - NF .. ty0 + RY + NF - 1,
    // periodic in y, one copy per contiguous run of rows; planes outside the grid
    // complete the stage's phase without a copy
    constexpr uint32_t row_bytes = NX * sizeof(C);
    auto issue = [&](int f, int q) {
        if (f < 0 || f >= nz) {
            mbar_arrive_expect_tx(&bar[q], 0u);
            return;
        }
        mbar_arrive_expect_tx(&bar[q], (PO ? 2u : 1u) * SR * row_bytes);
        C* sz = stages + q * STAGE;
        C* sp = sz + SLAB;
        fence_proxy_async_smem();
        int srow = 0;
        while (srow < SR) {
            int gy = (ty0 - NF + srow) % ny;
            if (gy < 0) gy += ny;
            const int n = min(SR - srow, ny - gy);
            const long long src = (long long)f * plane + (long long)gy * NX;
            bulk_g2s(sz + srow * NX, X + src, (uint32_t)n * row_bytes, &bar[q]);
            if (PO) bulk_g2s(sp + srow * NX, PO + src, (uint32_t)n * row_bytes, &bar[q]);
            srow += n;
        }
    };
    // ring slot of fill step j = f - f0 is j mod NR: the plane loop below is unrolled by
    // NR, so every slot index is a compile-time constant
    const int f0 = k0 - NF, f1 = k1 + NF;
    // ring slot u from stage q (zeros outside the grid), p of the own rows
    auto fill = [&](int f, int u, int q) {
        C* slot = ring + u * TILE;
        const bool in = f >= 0 && f < nz;
        const bool own_p = PN && f >= k0 && f < k1;
        const C* sz = stages + q * STAGE;
        const C* sp = sz + SLAB;
        C* pn = own_p ? PN + (long long)f * plane + (long long)ty0 * NX : nullptr;
#pragma unroll
        for (int it = 0; it < (SR * NX + NT - 1) / NT; ++it) {
            const int i = tid + it * NT;
            if ((SR * NX) % NT == 0 || i < SR * NX) {
                const int row = i / NX, col = i - row * NX;
                C v = czero<C>();
                if (in) {
                    v = sz[i];
                    if (PO) v = cfma(beta, sp[i], v);
                }
                C* trow = slot + row * TP;
                trow[NF + col] = v;
                if (col < NF) trow[NF + NX + col] = v;
                if (col >= NX - NF) trow[col - (NX - NF)] = v;
                if (own_p && row >= NF && row < NF + RY) pn[i - NF * NX] = v;
            }
        }
    };
    // a CTA barrier that also agrees on a failed wait; on failure the CTA drains the
    // copies it still has in flight (fill steps fw .. fw + D - 1) and the kernel returns
    auto barrier_ok = [&](bool ok, int fw) -> bool {
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                if (a.err) atomicExch(a.err, ERR_STAGE_TIMEOUT);
                for (int j = fw; j < fw + D && j < f1; ++j)
                    mbar_wait_bounded(&bar[(j - f0) % D], ((j - f0) / D) & 1);
            }
            __syncthreads();
            return false;
        }
        return true;
    };

    if (tid == 0)
        for (int j = 0; j < D && f0 + j < f1; ++j) issue(f0 + j, j);
    float dre = 0.f, dim = 0.f, nrm = 0.f;
    const int own = (NF + r) * TP + NF + x;
    const long long own_g = (long long)(ty0 + r) * NX + x;
    C* __restrict__ Yk = a.y + base + (long long)k0 * plane + own_g;
    const T* __restrict__ Vk = Vg ? Vg + (long long)k0 * plane + own_g : nullptr;
    bool failed = false;
    for (int f = f0; f < f1 && !failed; f += NR) {
#pragma unroll
        for (int u = 0; u < NR; ++u) {
            const int fu = f + u;
            if (fu >= f1) break;
            const int j = fu - f0;   // = (f - f0) + u with (f - f0) a multiple of NR
            constexpr int Dq = D;
            const int q = (NR % Dq == 0) ? (u % Dq) : (j % Dq);
            bool ok = mbar_wait_bounded(&bar[q], (j / Dq) & 1, wlim);
            if (j == 0 && a.wait_inject && tid == 0) ok = ok && mbar_wait_bounded(&bar[D], 0, wlim);
            fill(fu, u, q);
            if (!barrier_ok(ok, fu)) {
                failed = true;
                break;
            }
            if (tid == 0 && fu + D < f1) issue(fu + D, q);
            if (fu - NF < k0) continue;
            // output plane k = fu - N_f in slot (u - N_f) mod NR; every tap from the ring
            const C* c = ring + ((u - NF + NR) % NR) * TILE + own;
            const C x0 = *c;
            const T d = cen + a.vsign * (Vk ? *Vk : (T)0);
            C acc;
            if (a.iso) {
                const C x2 = p2add(x0, x0);
                C az = p2mul(x0, make_float2(d, d));
                C ax = make_float2(0.f, 0.f), ay = ax;
#pragma unroll
                for (int n = 1; n <= NF; ++n) {
                    const C cc = make_float2(a.cz[n], a.cz[n]);
                    const C zm = ring[((u - NF - n + 2 * NR) % NR) * TILE + own];
                    const C zp = ring[((u - NF + n + NR) % NR) * TILE + own];
                    az = p2fma(cc, p2sub(p2add(zm, zp), x2), az);
                    ax = p2fma(cc, p2sub(p2add(c[-n], c[n]), x2), ax);
                    ay = p2fma(cc, p2sub(p2add(c[-n * TP], c[n * TP]), x2), ay);
                }
                acc = p2add(az, p2add(ax, ay));
            } else {
                const C x2 = cadd(x0, x0);
                C az = cscale(x0, d);
                C ax = make_float2(0.f, 0.f), ay = ax;
#pragma unroll
                for (int n = 1; n <= NF; ++n) {
                    const C zm = ring[((u - NF - n + 2 * NR) % NR) * TILE + own];
                    const C zp = ring[((u - NF + n + NR) % NR) * TILE + own];
                    az = caxpy(a.cz[n], csub(cadd(zm, zp), x2), az);
                    ax = caxpy(a.cx[n], csub(cadd(c[-n], c[n]), x2), ax);
                    ay = caxpy(a.cy[n], csub(cadd(c[-n * TP], c[n * TP]), x2), ay);
                }
                acc = cadd(az, cadd(ax, ay));
            }
            *Yk = acc;
            Yk += plane;
            if (Vk) Vk += plane;
            if (a.dot_mode) {
                dre = fmaf(x0.x, acc.x, fmaf(-x0.y, acc.y, dre));
                dim = fmaf(x0.x, acc.y, fmaf(x0.y, acc.x, dim));
                nrm = fmaf(x0.x, x0.x, fmaf(x0.y, x0.y, nrm));
            }
        }
    }
    if (failed) return;

    if (a.dot_mode) {
        // partial slots are numbered per kRowTY-row tile (stencil_slots): the CTA's sum
        // goes to the first of its RY / kRowTY slots, zeros to the others
        static_assert(RY % kRowTY == 0, "RY spans whole row tiles");
        double r0d = dre, r1 = dim, r2 = nrm;
        block_reduce_3(r0d, r1, r2, red);
        if (tid < RY / kRowTY) {
            const int tiles_y = ny / kRowTY;
            const int slot = a.slot_base + blockIdx.x * (RY / kRowTY) + tid + blockIdx.y * tiles_y;
            a.dot_part[(long long)rhs * a.slot_stride + slot] =
                tid == 0 ? make_double2(r0d, r1) : make_double2(0.0, 0.0);
            if (a.nrm_part) a.nrm_part[(long long)rhs * a.slot_stride + slot] = tid == 0 ? r2 : 0.0;
        }
    }
}

static bool use_rows(int nx, int nf) { return nx >= nf && nx >= 4 && nx <= 64; }

// bulk-copy variant: FP32, rows of a multiple of 16 bytes, 16-byte aligned operands
static bool tma_width(int nx) {
    return nx == 12 || nx == 16 || nx == 24 || nx == 32 || nx == 48 || nx == 64;
}

template <typename T>
static bool use_rows_tma(const StencilArgs<T>& a) {
    if (sizeof(T) != 4 || (a.variant != 0 && a.variant != 3 && a.variant != 4) || !use_rows(a.nx, a.nf) ||
        !tma_width(a.nx))
        return false;
    uintptr_t al = reinterpret_cast<uintptr_t>(a.x);
    if (a.fused_p) al |= reinterpret_cast<uintptr_t>(a.pbufs[0]) | reinterpret_cast<uintptr_t>(a.pbufs[1]);
    return (al & 15) == 0;
}

template <int NX, int NF>
static cudaError_t prepare_tma() {
    constexpr int MB = NX * kRowTY <= 384 ? 3 : 2;
    cudaError_t e = cudaFuncSetAttribute(k_stencil_rows_tma<NX, NF, MB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)RowsTma<NX, NF>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stencil_rows_tma<NX, NF, MB>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

// row-blocked kernel shape: PT rows per thread, TY thread rows (RY = 16 own rows)
template <int NX> struct BlkShape {
    static constexpr int PT = 4;
    static constexpr int TY = 16 / PT;
    static constexpr int MINB = 2;
    static constexpr int D = 3;
};

template <int NX, int NF>
static cudaError_t prepare_blk() {
    using S = BlkShape<NX>;
    cudaError_t e = cudaFuncSetAttribute(k_stencil_blk<NX, NF, S::PT, S::TY, S::MINB, S::D>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BlkTma<NX, NF, S::PT, S::TY, S::D>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stencil_blk<NX, NF, S::PT, S::TY, S::MINB, S::D>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

// the blocked kernel: FP32 bulk-copy rows, N_f 1 (Eq. 10) or 4 (the operator), whole
// 16-row tiles in y, the fastest-kernel variant
template <typename T>
static bool use_blk(const StencilArgs<T>& a) {
    return a.variant == 0 && (a.nf == 1 || a.nf == 4) && a.ny % 16 == 0 && a.nx >= 2 * a.nf;
}

template <int NX, int NF>
static void launch_blk(const StencilArgs<float>& a, dim3 grid, cudaStream_t s) {
    using S = BlkShape<NX>;
    k_stencil_blk<NX, NF, S::PT, S::TY, S::MINB, S::D>
        <<<grid, NX * S::TY, BlkTma<NX, NF, S::PT, S::TY, S::D>::smem, s>>>(a);
}

template <int NX>
static cudaError_t launch_blk_nf(const StencilArgs<float>& a, int nrhs, cudaStream_t s) {
    const int nzc = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(a.ny / 16, nzc, nrhs);
    switch (a.nf) {
        case 1: launch_blk<NX, 1>(a, grid, s); break;
        case 4: launch_blk<NX, 4>(a, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NX, int NF>
static cudaError_t prepare_ring() {
    return cudaFuncSetAttribute(k_stencil_ring<NX, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RingTma<NX, NF>::smem);
}

// the ring kernel: FP32 bulk-copy rows, N_f 1 or 4, whole 16-row tiles in y
template <typename T>
static bool use_ring(const StencilArgs<T>& a) {
    return a.variant == 4 && (a.nf == 1 || a.nf == 4) && a.ny % 16 == 0 && a.nx >= 2 * a.nf;
}

template <int NX>
static cudaError_t launch_ring_nf(const StencilArgs<float>& a, int nrhs, cudaStream_t s) {
    const int nzc = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(a.ny / 16, nzc, nrhs);
    switch (a.nf) {
        case 1: k_stencil_ring<NX, 1><<<grid, NX * 16, RingTma<NX, 1>::smem, s>>>(a); break;
        case 4: k_stencil_ring<NX, 4><<<grid, NX * 16, RingTma<NX, 4>::smem, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int NX>
static cudaError_t prepare_tma_nf() {
    cudaError_t e = prepare_tma<NX, 1>();
    if (e == cudaSuccess) e = prepare_tma<NX, 2>();
    if (e == cudaSuccess) e = prepare_tma<NX, 3>();
    if (e == cudaSuccess) e = prepare_tma<NX, 4>();
    if (e == cudaSuccess && NX >= 2) e = prepare_blk<NX, 1>();
    if (e == cudaSuccess && NX >= 8) e = prepare_blk<NX, 4>();
    if (e == cudaSuccess && NX >= 2) e = prepare_ring<NX, 1>();
    if (e == cudaSuccess && NX >= 8) e = prepare_ring<NX, 4>();
    return e;
}

cudaError_t stencil_prepare() {
    cudaError_t e = prepare_tma_nf<12>();
    if (e == cudaSuccess) e = prepare_tma_nf<16>();
    if (e == cudaSuccess) e = prepare_tma_nf<24>();
    if (e == cudaSuccess) e = prepare_tma_nf<32>();
    if (e == cudaSuccess) e = prepare_tma_nf<48>();
    if (e == cudaSuccess) e = prepare_tma_nf<64>();
    return e;
}

template <int NX, int NF>
static void launch_tma(const StencilArgs<float>& a, dim3 grid, cudaStream_t s) {
    constexpr int MB = NX * kRowTY <= 384 ? 3 : 2;
    k_stencil_rows_tma<NX, NF, MB><<<grid, NX * kRowTY, RowsTma<NX, NF>::smem, s>>>(a);
}

template <int NX>
static cudaError_t launch_tma_nf(const StencilArgs<float>& a, dim3 grid, cudaStream_t s) {
    switch (a.nf) {
        case 1: launch_tma<NX, 1>(a, grid, s); break;
        case 2: launch_tma<NX, 2>(a, grid, s); break;
        case 3: launch_tma<NX, 3>(a, grid, s); break;
        case 4: launch_tma<NX, 4>(a, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stencil(const StencilArgs<T>& a0, int nrhs, cudaStream_t s) {
    if constexpr (sizeof(T) == 8) {
        if (a0.variant == 2 && !a0.fused_p && !a0.dot_mode && !a0.rhs_sign &&
            stencil_df_supported(a0.nx, a0.nf))
            return launch_stencil_df(a0, nrhs, s);
    }
    if (use_rows(a0.nx, a0.nf)) {
        StencilArgs<T> a = a0;
        if (a.zchunk <= 0) a.zchunk = 32;
        a.tiles_x = 1;
        a.tiles_y = (a.ny + kRowTY - 1) / kRowTY;
        const int nzc = (a.nz + a.zchunk - 1) / a.zchunk;
        dim3 grid(a.tiles_y, nzc, nrhs);
        const int threads = a.nx * kRowTY;
        using C = typename Cplx<T>::type;
        if constexpr (sizeof(T) == 4) {
            if (use_rows_tma(a) && use_ring(a)) {
                switch (a.nx) {
                    case 12: return launch_ring_nf<12>(a, nrhs, s);
                    case 16: return launch_ring_nf<16>(a, nrhs, s);
                    case 24: return launch_ring_nf<24>(a, nrhs, s);
                    case 32: return launch_ring_nf<32>(a, nrhs, s);
                    case 48: return launch_ring_nf<48>(a, nrhs, s);
                    case 64: return launch_ring_nf<64>(a, nrhs, s);
                    default: return cudaErrorInvalidValue;
                }
            }
            if (use_rows_tma(a) && use_blk(a)) {
                switch (a.nx) {
                    case 12: return launch_blk_nf<12>(a, nrhs, s);
                    case 16: return launch_blk_nf<16>(a, nrhs, s);
                    case 24: return launch_blk_nf<24>(a, nrhs, s);
                    case 32: return launch_blk_nf<32>(a, nrhs, s);
                    case 48: return launch_blk_nf<48>(a, nrhs, s);
                    case 64: return launch_blk_nf<64>(a, nrhs, s);
                    default: return cudaErrorInvalidValue;
                }
            }
            if (use_rows_tma(a)) {
                switch (a.nx) {
                    case 12: return launch_tma_nf<12>(a, grid, s);
                    case 16: return launch_tma_nf<16>(a, grid, s);
                    case 24: return launch_tma_nf<24>(a, grid, s);
                    case 32: return launch_tma_nf<32>(a, grid, s);
                    case 48: return launch_tma_nf<48>(a, grid, s);
                    case 64: return launch_tma_nf<64>(a, grid, s);
                    default: return cudaErrorInvalidValue;
                }
            }
        }
        const size_t smem = sizeof(C) * (size_t)(kRowTY + 2 * a.nf) * a.nx;
        switch (a.nf) {
            case 1: k_stencil_rows<T, 1><<<grid, threads, smem, s>>>(a); break;
            case 2: k_stencil_rows<T, 2><<<grid, threads, smem, s>>>(a); break;
            case 3: k_stencil_rows<T, 3><<<grid, threads, smem, s>>>(a); break;
            case 4: k_stencil_rows<T, 4><<<grid, threads, smem, s>>>(a); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    return launch_stencil_tiles<T>(a0, nrhs, s);
}

template <typename T>
cudaError_t launch_stencil_tiles(const StencilArgs<T>& a0, int nrhs, cudaStream_t s) {
    StencilArgs<T> a = a0;
    a.tiles_x = (a.nx + kTX - 1) / kTX;
    a.tiles_y = (a.ny + kTY - 1) / kTY;
    if (a.zchunk <= 0) a.zchunk = 32;
    const int nzc = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(a.tiles_x * a.tiles_y, nzc, nrhs);
    dim3 block(kTX, kTY);
    switch (a.nf) {
        case 1: k_stencil<T, 1><<<grid, block, 0, s>>>(a); break;
        case 2: k_stencil<T, 2><<<grid, block, 0, s>>>(a); break;
        case 3: k_stencil<T, 3><<<grid, block, 0, s>>>(a); break;
        case 4: k_stencil<T, 4><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// number of dot slots a stencil launch writes per RHS (nf: taps of that launch;
// the preconditioner (nf = 1) and the operator use the same tiling for the same
// lateral size as long as use_rows agrees, which holds for nx >= 4)
int stencil_slots(int nx, int ny, int nz, int zchunk, int nf) {
    if (zchunk <= 0) zchunk = 32;
    const int nzc = (nz + zchunk - 1) / zchunk;
    if (use_rows(nx, nf)) return ((ny + kRowTY - 1) / kRowTY) * nzc;
    return ((nx + kTX - 1) / kTX) * ((ny + kTY - 1) / kTY) * nzc;
}

template cudaError_t launch_stencil<float>(const StencilArgs<float>&, int, cudaStream_t);
template cudaError_t launch_stencil<double>(const StencilArgs<double>&, int, cudaStream_t);

}  // namespace iobm
