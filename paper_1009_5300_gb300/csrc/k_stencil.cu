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

namespace iobm {

constexpr int kTX = 32;
constexpr int kTY = 8;

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
#pragma unroll
                for (int n = 1; n <= NF; ++n) {
                    acc = caxpy(a.cz[n], cadd(q[NF - n], q[NF + n]), acc);
                    acc = caxpy(a.cx[n], cadd(tile[ly + NF][lx + NF - n], tile[ly + NF][lx + NF + n]), acc);
                    acc = caxpy(a.cy[n], cadd(tile[ly + NF - n][lx + NF], tile[ly + NF + n][lx + NF]), acc);
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
#pragma unroll
                for (int n = 1; n <= NF; ++n) {
                    const int xm = (x - n < 0) ? x - n + nx : x - n;
                    const int xp = (x + n >= nx) ? x + n - nx : x + n;
                    acc = caxpy(a.cz[n], cadd(q[NF - n], q[NF + n]), acc);
                    acc = caxpy(a.cx[n], cadd(row[xm], row[xp]), acc);
                    acc = caxpy(a.cy[n], cadd(row[x - n * nx], row[x + n * nx]), acc);
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

static bool use_rows(int nx, int nf) { return nx >= nf && nx >= 4 && nx <= 64; }

template <typename T>
cudaError_t launch_stencil(const StencilArgs<T>& a0, int nrhs, cudaStream_t s) {
    if (use_rows(a0.nx, a0.nf)) {
        StencilArgs<T> a = a0;
        if (a.zchunk <= 0) a.zchunk = 32;
        a.tiles_x = 1;
        a.tiles_y = (a.ny + kRowTY - 1) / kRowTY;
        const int nzc = (a.nz + a.zchunk - 1) / a.zchunk;
        dim3 grid(a.tiles_y, nzc, nrhs);
        const int threads = a.nx * kRowTY;
        using C = typename Cplx<T>::type;
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
