// The FP64 solve: one kernel per stage of Sec. 5.2.2 plus the near field,
// the gauge and the energy, and the plan / solve entry points of dpslab.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "kernels.cuh"
#include "zgemm.cuh"

using namespace dps;

namespace {

constexpr int kColBlock = 4;        // k_par columns per block of the column kernel (one warp each)
constexpr int kColThreads = 32 * kColBlock;
constexpr int kChargeThreads = 256;
constexpr int kInterpWarps = 2;     // default warps per block of the interpolation (one charge each)
constexpr int kMaxInterpWarps = 8;
constexpr int kTile = 16;           // spreading tile: kTile x kTile xy grid points, one thread each
constexpr int kSpreadBatch = 32;    // sources per batch in the tiled spreading
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kStageNear = 10;      // index of the near stage in the stage timings (dpslab_stage_name)

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of V = 2^k values at once (transposed butterfly): at each of the
// first k steps a lane keeps half of its values and sends the other half to
// its partner, which adds them to its own; the last 5 - k steps are plain.
// That is V - 1 + 5 - k shuffles instead of 5 V. On return lane l holds the
// sum of value (l >> (5 - k)) & (V - 1).
template <int V, class T>
__device__ __forceinline__ T warp_sum_multi(const T* in) {
    static_assert(V >= 1 && V <= 32 && (V & (V - 1)) == 0, "V is a power of two up to 32");
    T a[V];
#pragma unroll
    for (int i = 0; i < V; ++i) a[i] = in[i];
    const int lane = threadIdx.x & 31;
    int o = 16;
#pragma unroll
    for (int h = V / 2; h >= 1; h /= 2, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = up ? a[i] : a[i + h];
            const T keep = up ? a[i + h] : a[i];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    T r = a[0];
#pragma unroll
    for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; result valid in thread 0. All threads must call it.
__device__ double block_sum(double v) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

// The column stage of up to kBatchMaxSys systems in one launch: their
// parameter blocks travel as the kernel's (read-only) parameter, 32 KB at
// most, so that the kernels read them as they read a single system's.
constexpr int kBatchMaxSys = 21;
constexpr int kMaxOPairs = 32;      // node pairs of rho_o transformed in the column kernel (else by the z GEMM)
struct ColBatch {
    int nsys;
    int starts[kBatchMaxSys + 1];        // first column block of each system
    KP kp[kBatchMaxSys];
};
static_assert(sizeof(ColBatch) <= 32000, "kernel parameters are limited to 32 KB");

// System of block b of a launch over several systems: starts[s] is the
// first block of system s (ascending, starts[0] = 0); the largest s with
// starts[s] <= b.
__device__ __forceinline__ int batch_system(const int* starts, int nsys, int b) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Cell list index, z fastest: the cell-sorted charge order then sweeps thin
// y-slabs of the box, whose grid neighbourhood stays in L2 while the
// interpolation gathers from it.
__device__ __forceinline__ int cell_index(const KP& kp, int cx, int cy, int cz) {
    return (cy * kp.ncx + cx) * kp.ncz + cz;
}

__device__ __forceinline__ int wrap_index(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// ---------------------------------------------------------------------------
// charges: validation, wrapping, neutrality sums, cell histogram
// ---------------------------------------------------------------------------
__global__ void k_prepare(KP kp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double qv = 0.0, aq = 0.0;
    if (k < kp.n) {
        double x = kp.pos[3 * k], y = kp.pos[3 * k + 1], z = kp.pos[3 * k + 2], q = kp.q[k];
        int bad = 0;
        if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(q)) bad = kStatusNonFinite;
        else if (!(z > 0.0 && z < kp.H)) bad = kStatusOutOfSlab;
        if (bad) {
            atomicOr(kp.status, bad);
            x = 0.0; y = 0.0; z = 0.5 * kp.H; q = 0.0;
        }
        x = np_mod(x, kp.Lx);
        y = np_mod(y, kp.Ly);
        kp.part[k] = make_double4_32a(x, y, z, q);
        qv = q;
        aq = fabs(q);
        if (kp.near_on) {
            const int cx = min(kp.ncx - 1, max(0, int(x / kp.cwx)));
            const int cy = min(kp.ncy - 1, max(0, int(y / kp.cwy)));
            const int cz = min(kp.ncz - 1, max(0, int(z / kp.cwz)));
            const int c = cell_index(kp, cx, cy, cz);
            kp.cell_of[k] = c;
            atomicAdd(&kp.cell_count[c], 1);
        }
    }
    const double s1 = block_sum(qv);
    const double s2 = block_sum(aq);
    if (threadIdx.x == 0) {
        kp.part_q[blockIdx.x] = s1;
        kp.part_q[gridDim.x + blockIdx.x] = s2;
    }
}

// Multi-block exclusive scan of count[0..n) into start[0..n]: block sums of
// kScanChunk elements, a one-block scan of those sums (k_scan), then each
// block scans its chunk and adds its offset.
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanBlock * kScanItems;

__global__ void __launch_bounds__(kScanBlock) k_scan_sums(const int* count, int n, int* part) {
    __shared__ int red[32];
    const int base = blockIdx.x * kScanChunk;
    int s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        const int idx = base + i * kScanBlock + threadIdx.x;
        if (idx < n) s += count[idx];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = red[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_apply(const int* count, int* start, int n, const int* offs) {
    __shared__ int red[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int base = blockIdx.x * kScanChunk + tid * kScanItems;
    int v[kScanItems], t = 0;
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? count[base + i] : 0;
        t += v[i];
    }
    int inc = t;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) red[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = red[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        red[lane] = w;
    }
    __syncthreads();
    int run = offs[blockIdx.x] + (warp ? red[warp - 1] : 0) + inc - t;
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) start[base + i] = run;
        run += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && tid == 0) start[n] = offs[gridDim.x];
}

// exclusive scan of count[0..n) into start[0..n], one block of 1024 threads
__global__ void k_scan(const int* count, int* start, int n) {
    __shared__ int sums[1024];
    const int tid = threadIdx.x, bs = blockDim.x;
    const int chunk = (n + bs - 1) / bs;
    const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += count[i];
    sums[tid] = s;
    __syncthreads();
    for (int o = 1; o < bs; o <<= 1) {
        const int v = tid >= o ? sums[tid - o] : 0;
        __syncthreads();
        sums[tid] += v;
        __syncthreads();
    }
    int run = sums[tid] - s;
    for (int i = lo; i < hi; ++i) {
        start[i] = run;
        run += count[i];
    }
    if (tid == bs - 1) start[n] = sums[bs - 1];
}

// Nodes j with |z_j - z| <= H_E (the nodes descend in j): first an estimate
// from arccos, then the exact test on the node values.
__device__ __forceinline__ void node_range(const KP& kp, double z, int& j0, int& j1) {
    const int N = kp.nz;
    const double sc = double(N - 1) / 3.14159265358979323846;
    auto jof = [&](double zz) {
        const double sv = fmin(1.0, fmax(-1.0, 2.0 * (zz - kp.a) / kp.Hbar - 1.0));
        return acos(sv) * sc;
    };
    j0 = max(0, int(floor(jof(z + kp.HE))) - 1);
    j1 = min(N - 1, int(ceil(jof(z - kp.HE))) + 1);
    while (j0 <= j1 && kp.zn[j0] - z > kp.HE) ++j0;
    while (j1 >= j0 && z - kp.zn[j1] > kp.HE) --j1;
    // the estimate brackets the range; widen if rounding cut it
    while (j0 > 0 && fabs(kp.zn[j0 - 1] - z) <= kp.HE) --j0;
    while (j1 < N - 1 && fabs(kp.zn[j1 + 1] - z) <= kp.HE) ++j1;
}

// Source s (0: the charge, 1: its image below z = 0, 2: above z = H) of
// charge p, Sec. 5.2.2 step 1 and Eq. (ims); false if it does not exist.
__device__ __forceinline__ bool make_source(const KP& kp, const double4_32a& p, int s, SrcRec& r, int& tile) {
    double z = p.z, q = p.w;
    const bool nb = p.z <= 2.0 * kp.HE, nt = p.z >= kp.H - 2.0 * kp.HE;
    if (s == 1) {
        if (!nb || kp.Gb == 0.0) return false;
        z = -p.z; q = -kp.Gb * p.w;
    } else if (s == 2) {
        if (!nt || kp.Gt == 0.0) return false;
        z = 2.0 * kp.H - p.z; q = -kp.Gt * p.w;
    }
    const double HE = kp.HE;
    r.z = z;
    r.q = q;
    r.xlo = int(ceil((p.x - HE) / kp.hx));
    r.ylo = int(ceil((p.y - HE) / kp.hy));
    r.sx = int(floor((p.x + HE) / kp.hx)) - r.xlo + 1;
    r.sy = int(floor((p.y + HE) / kp.hy)) - r.ylo + 1;
    r.d0x = double(r.xlo) * kp.hx - p.x;
    r.d0y = double(r.ylo) * kp.hy - p.y;
    node_range(kp, z, r.j0, r.j1);
    r.over = (s == 0) && (nb || nt);
    r.pad = 0;
    const int tx = min(kp.ntx - 1, int(floor(p.x / kp.hx)) / kTile);
    const int ty = min(kp.nty - 1, int(floor(p.y / kp.hy)) / kTile);
    tile = ty * kp.ntx + tx;
    return r.j0 <= r.j1 && q != 0.0;
}

__global__ void k_count_sources(KP kp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kp.n) return;
    const double4_32a p = kp.part[k];
    for (int s = 0; s < 3; ++s) {
        SrcRec r;
        int tile;
        if (!make_source(kp, p, s, r, tile)) continue;
        for (int sl = r.j0 / kp.slab; sl <= r.j1 / kp.slab; ++sl) atomicAdd(&kp.tile_count[sl * kp.ntiles + tile], 1);
    }
}

__global__ void k_scatter_sources(KP kp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kp.n) return;
    const double4_32a p = kp.part[k];
    for (int s = 0; s < 3; ++s) {
        SrcRec r;
        int tile;
        if (!make_source(kp, p, s, r, tile)) continue;
        for (int sl = r.j0 / kp.slab; sl <= r.j1 / kp.slab; ++sl) {
            const int b = sl * kp.ntiles + tile;
            kp.srcs[kp.tile_start[b] + atomicAdd(&kp.tile_fill[b], 1)] = r;
        }
    }
}

// ---------------------------------------------------------------------------
// spreading, Sec. 5.2.2 steps 2-3, output-stationary: block (tile, z slab)
// owns kTile x kTile grid columns (one thread each) and kp.slab z nodes, and
// sums every source of the neighbouring tiles into shared memory; each grid
// point is written once. rho_i gets every source, rho_o only charges of
// C_over (z within 2 H_E of a wall; images lie outside 0 < z < H). The
// support is the closed box |dx|, |dy|, |dz| <= H_E with the same index rule
// ceil((x - H_E)/h) .. floor((x + H_E)/h) as a direct scatter.
// ---------------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(kTile * kTile) k_spread_tiled(KP kp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int B = kSpreadBatch;
    const int SZ = kp.slab;
    const int TX = (kp.supx + 31) & ~31, TY = (kp.supy + 31) & ~31;   // table strides
    R* acc_i = reinterpret_cast<R*>(smraw);                 // [SZ][256]
    R* acc_o = acc_i + SZ * kTile * kTile;                   // [SZ][256]
    R* wxt = acc_o + SZ * kTile * kTile;                     // [B][TX]
    R* wyt = wxt + B * TX;                                   // [B][TY]
    R* wzt = wyt + B * TY;                                   // [B][SZ]
    __shared__ int s_dx0[B], s_dy0[B], s_sx[B], s_sy[B], s_z0[B], s_z1[B], s_over[B], s_ok[B];
    __shared__ R s_q[B];
    __shared__ double s_d0x[B], s_d0y[B], s_zs[B];
    __shared__ int s_tiles[64], s_pre[65];
    __shared__ unsigned s_mx[kTile], s_my[kTile];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x, txi = tile % kp.ntx, tyi = tile / kp.ntx;
    const int slab = blockIdx.y;
    const int js = slab * SZ, je = min(kp.nz, js + SZ);
    const int gx0 = txi * kTile, gy0 = tyi * kTile;
    const int tw = min(kp.nx, gx0 + kTile) - gx0, th = min(kp.ny, gy0 + kTile) - gy0;
    const int lx = tid % kTile, ly = tid / kTile;
    const int gx = gx0 + lx, gy = gy0 + ly;
    const bool mine = lx < tw && ly < th;
    for (int i = tid; i < 2 * SZ * kTile * kTile; i += blockDim.x) acc_i[i] = R(0);
    if (tid == 0) {
        const int r = kp.tile_r;
        const int nxs = min(2 * r + 1, kp.ntx), nys = min(2 * r + 1, kp.nty);
        int cnt = 0, run = 0;
        for (int oy = 0; oy < nys; ++oy) {
            const int ty = nys == kp.nty ? oy : wrap_index(tyi - r + oy, kp.nty);
            for (int ox = 0; ox < nxs; ++ox) {
                const int tx = nxs == kp.ntx ? ox : wrap_index(txi - r + ox, kp.ntx);
                const int bk = slab * kp.ntiles + ty * kp.ntx + tx;
                s_tiles[cnt] = bk;
                s_pre[cnt] = run;
                run += kp.tile_start[bk + 1] - kp.tile_start[bk];
                ++cnt;
            }
        }
        s_pre[cnt] = run;
        s_tiles[63] = cnt;
    }
    __syncthreads();
    const int ntl = s_tiles[63], total = s_pre[ntl];
    const R ig2 = R(1.0 / (2.0 * kp.gt * kp.gt));
    const R s1 = R(kp.s1norm);
    for (int base = 0; base < total; base += B) {
        // phase 1: warp 0, one lane per source of the batch; then the
        // coverage masks, transposed with ballots: bit b of s_mx[lx] says
        // source b covers tile column lx (likewise s_my[ly] for rows)
        if (tid < B) {
            const int c = base + tid;
            int ok = 0;
            unsigned xm = 0u, ym = 0u;
            if (c < total) {
                int t = 0;
                while (s_pre[t + 1] <= c) ++t;
                const SrcRec r = kp.srcs[kp.tile_start[s_tiles[t]] + (c - s_pre[t])];
                // offset of the tile's first column/row within the support (mod n)
                const int dx0 = wrap_index(gx0 - r.xlo, kp.nx), dy0 = wrap_index(gy0 - r.ylo, kp.ny);
                for (int l = 0; l < tw; ++l) {
                    int i = dx0 + l;
                    if (i >= kp.nx) i -= kp.nx;
                    if (i < r.sx) xm |= 1u << l;
                }
                for (int l = 0; l < th; ++l) {
                    int i = dy0 + l;
                    if (i >= kp.ny) i -= kp.ny;
                    if (i < r.sy) ym |= 1u << l;
                }
                const int z0 = max(r.j0, js), z1 = min(r.j1, je - 1);
                ok = xm && ym && z0 <= z1;
                s_dx0[tid] = dx0; s_dy0[tid] = dy0; s_sx[tid] = r.sx; s_sy[tid] = r.sy;
                s_z0[tid] = z0; s_z1[tid] = z1; s_over[tid] = r.over; s_q[tid] = R(r.q);
                s_d0x[tid] = r.d0x; s_d0y[tid] = r.d0y; s_zs[tid] = r.z;
            }
            s_ok[tid] = ok;
            if (!ok) { xm = 0u; ym = 0u; }
            for (int l = 0; l < kTile; ++l) {
                const unsigned bx = __ballot_sync(0xffffffffu, (xm >> l) & 1u);
                const unsigned by = __ballot_sync(0xffffffffu, (ym >> l) & 1u);
                if (tid == 0) { s_mx[l] = bx; s_my[l] = by; }
            }
        }
        __syncthreads();
        // phase 2: warp w fills the weight tables of sources w, w + 8, ...
        // (offset d = d0 + i h, d0 taken in double per source)
        for (int b = warp; b < B; b += (kTile * kTile) / 32) {
            if (!s_ok[b]) continue;
            const R d0x = R(s_d0x[b]), d0y = R(s_d0y[b]);
            for (int i = lane; i < s_sx[b]; i += 32) {
                const R d = d0x + R(i) * R(kp.hx);
                wxt[b * TX + i] = s1 * dexp(-d * d * ig2);
            }
            for (int i = lane; i < s_sy[b]; i += 32) {
                const R d = d0y + R(i) * R(kp.hy);
                wyt[b * TY + i] = s1 * dexp(-d * d * ig2);
            }
            for (int i = lane; i <= s_z1[b] - s_z0[b]; i += 32) {
                const R d = R(kp.zn[s_z0[b] + i] - s_zs[b]);
                wzt[b * SZ + i] = s1 * dexp(-d * d * ig2);
            }
        }
        __syncthreads();
        // phase 3: the warp walks the union of its lanes' covering sources
        // (uniform loop, broadcast loads); each covered lane adds its column
        {
            const unsigned mine_hits = mine ? (s_mx[lx] & s_my[ly]) : 0u;
            unsigned hits = __reduce_or_sync(0xffffffffu, mine_hits);
            while (hits) {
                const int b = __ffs(hits) - 1;
                hits &= hits - 1u;
                if (!((mine_hits >> b) & 1u)) continue;
                int ix = s_dx0[b] + lx;
                if (ix >= kp.nx) ix -= kp.nx;
                int iy = s_dy0[b] + ly;
                if (iy >= kp.ny) iy -= kp.ny;
                const R w = s_q[b] * wxt[b * TX + ix] * wyt[b * TY + iy];
                const int z0 = s_z0[b], z1 = s_z1[b];
                const R* wz = wzt + b * SZ - z0;
                R* ai = acc_i + (z0 - js) * kTile * kTile + tid;
                if (s_over[b]) {
                    R* ao = acc_o + (z0 - js) * kTile * kTile + tid;
                    for (int j = z0; j <= z1; ++j, ai += kTile * kTile, ao += kTile * kTile) {
                        const R v = w * wz[j];
                        *ai += v;
                        *ao += v;
                    }
                } else {
                    for (int j = z0; j <= z1; ++j, ai += kTile * kTile) *ai += w * wz[j];
                }
            }
        }
        __syncthreads();
    }
    if (mine) {
        R* rho = static_cast<R*>(kp.rho);
        const size_t G = size_t(kp.nz) * kp.ny * kp.nx;
        for (int j = js; j < je; ++j) {
            const size_t g = (size_t(j) * kp.ny + gy) * kp.nx + gx;
            rho[g] = acc_i[(j - js) * kTile * kTile + tid];
            rho[G + g] = acc_o[(j - js) * kTile * kTile + tid];
        }
    }
}

// ---------------------------------------------------------------------------
// spreading, mixed precision (Sec. 5.2.2 steps 2-3, same support rule as
// above): each source is stored in every (tile, slab) block it touches, so a
// block reads exactly the sources that reach it. The block's 256 threads own
// its 16 x 16 grid columns and keep their kSlabM z values of rho_i and rho_o
// in registers; per batch of sources the threads first fill the separable
// weight tables (x, y, and z times the strength) in shared memory.
// ---------------------------------------------------------------------------
constexpr int kSlabM = 8;
constexpr int kSpreadBatchM = 128;
constexpr int kWzStride = 12;      // z-table row stride (16-byte rows, fewer bank conflicts)

// Distinct tiles along one axis touched by support indices lo .. lo + s - 1
// (wrapped mod n; s <= n); returns their number (<= 6 for s < 64).
__device__ __forceinline__ int axis_tiles(int lo, int s, int n, int* out) {
    int col = wrap_index(lo, n), rem = s, cnt = 0;
    while (rem > 0) {
        const int t = col / kTile;
        const int take = min(rem, min(n, (t + 1) * kTile) - col);
        bool dup = false;
        for (int i = 0; i < cnt; ++i) dup |= out[i] == t;
        if (!dup) out[cnt++] = t;
        rem -= take;
        col += take;
        if (col >= n) col -= n;
    }
    return cnt;
}

// Node range |z_j - z| <= H_E (same rule and result as node_range): an
// arccos estimate, then the membership test in float on z and z_j as float
// pairs, falling back to the double test only within 1e-5 H_E of the edge.
__device__ __forceinline__ void node_range_f(const KP& kp, double z, float zhi, float zlo, int& j0, int& j1) {
    const int N = kp.nz;
    const float HE = kp.f.HE, sc = float(N - 1) * 0.318309886183790672f;
    auto jof = [&](float zz) {
        const float sv = fminf(1.f, fmaxf(-1.f, (zz - kp.f.a) * kp.f.sz - 1.f));
        return acosf(sv) * sc;
    };
    auto inside = [&](int j) -> bool {
        const float d = fabsf((kp.zn32[j] - zhi) + (kp.znlo32[j] - zlo));
        if (fabsf(d - HE) > 1e-5f * HE) return d <= HE;
        return fabs(kp.zn[j] - z) <= kp.HE;
    };
    j0 = max(0, int(floorf(jof(zhi + HE))) - 1);
    j1 = min(N - 1, int(ceilf(jof(zhi - HE))) + 1);
    while (j0 <= j1 && !inside(j0)) ++j0;
    while (j1 >= j0 && !inside(j1)) --j1;
    while (j0 > 0 && inside(j0 - 1)) --j0;
    while (j1 < N - 1 && inside(j1 + 1)) ++j1;
}

// Support window of a point in x or y: first index ceil((x - H_E)/h), size,
// and the float offset of the first index (double arithmetic).
__device__ __forceinline__ void axis_window(double x, double HE, double h, int& lo, int& sz, float& d0) {
    lo = int(ceil((x - HE) / h));
    sz = int(floor((x + HE) / h)) - lo + 1;
    d0 = float(double(lo) * h - x);
}

// Bucket counters shared by the lanes that call together: one atomic per
// distinct bucket b among them, adding the number of lanes with that b.
// agg_claim returns the lane's own slot (the counter's old value plus the
// lane's rank among those lanes).
__device__ __forceinline__ void agg_count(int* count, int b) {
    const unsigned peers = __match_any_sync(__activemask(), b);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(count + b, __popc(peers));
}
__device__ __forceinline__ int agg_claim(int* fill, int b) {
    const unsigned peers = __match_any_sync(__activemask(), b);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int old = 0;
    if (lane == leader) old = atomicAdd(fill + b, __popc(peers));
    return __shfl_sync(peers, old, leader) + __popc(peers & ((1u << lane) - 1u));
}

// One thread per charge, in cell-list order when there is one (slot i holds
// charge sorted_idx[i]; neighbouring threads then touch mostly the same
// buckets and share their atomics): the interpolation window of the charge
// (irec[i]), its spreading sources (the charge and its images, Eq. (ims)) as
// records srcs_tmp[3i + s], and the bucket counts of every (tile, slab)
// block each source touches.
__global__ void k_sources_f(KP kp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kp.n) return;
    const double4_32a p = kp.near_on ? kp.sorted[k] : kp.part[k];
    SrcF r;
    int sx, sy;
    axis_window(p.x, kp.HE, kp.hx, r.xlo, sx, r.d0x);
    axis_window(p.y, kp.HE, kp.hy, r.ylo, sy, r.d0y);
    const bool nb = p.z <= 2.0 * kp.HE, nt = p.z >= kp.H - 2.0 * kp.HE;
    int tx[6], ty[6];
    const int ntx = axis_tiles(r.xlo, sx, kp.nx, tx);
    const int nty = axis_tiles(r.ylo, sy, kp.ny, ty);
    for (int s = 0; s < 3; ++s) {
        double z = p.z, q = p.w;
        bool exists = true;
        if (s == 1) { exists = nb && kp.Gb != 0.0; z = -p.z; q = -kp.Gb * p.w; }
        if (s == 2) { exists = nt && kp.Gt != 0.0; z = 2.0 * kp.H - p.z; q = -kp.Gt * p.w; }
        unsigned pack = 0u;
        if (exists) {
            r.zhi = float(z);
            r.zlo = float(z - double(r.zhi));
            r.q = float(q);
            int j0, j1;
            node_range_f(kp, z, r.zhi, r.zlo, j0, j1);
            if (s == 0) {
                IRec ir;
                ir.d0x = r.d0x; ir.d0y = r.d0y; ir.zhi = r.zhi; ir.zlo = r.zlo;
                ir.xlo = r.xlo; ir.ylo = r.ylo;
                ir.sx = short(sx); ir.sy = short(sy); ir.j0 = short(j0); ir.j1 = short(j1);
                kp.irec[k] = ir;
            }
            if (j0 <= j1 && q != 0.0) {
                const unsigned over = (s == 0) && (nb || nt);
                pack = unsigned(sx) | (unsigned(sy) << 6) | (unsigned(j0) << 12) | (unsigned(j1) << 21) | (over << 30) |
                       (1u << 31);
                for (int sl = j0 / kSlabM; sl <= j1 / kSlabM; ++sl)
                    for (int a = 0; a < nty; ++a)
                        for (int c = 0; c < ntx; ++c) agg_count(kp.tile_count, sl * kp.ntiles + ty[a] * kp.ntx + tx[c]);
            }
        }
        r.pack = pack;
        kp.srcs_tmp[3 * size_t(k) + s] = r;
    }
}

__global__ void k_scatter_sources_f(KP kp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kp.n) return;
    int tx[6], ty[6], ntx = 0, nty = 0;
    for (int s = 0; s < 3; ++s) {
        const SrcF r = kp.srcs_tmp[3 * size_t(k) + s];
        if (!(r.pack >> 31)) continue;
        if (!ntx) {
            ntx = axis_tiles(r.xlo, r.pack & 63, kp.nx, tx);
            nty = axis_tiles(r.ylo, (r.pack >> 6) & 63, kp.ny, ty);
        }
        const int j0 = (r.pack >> 12) & 511, j1 = (r.pack >> 21) & 511;
        // per slab, up to 3 x 3 tiles at a time: every slot is claimed (the
        // atomics are independent) before the first record is stored, so
        // their round trips overlap
        for (int sl = j0 / kSlabM; sl <= j1 / kSlabM; ++sl)
            for (int a0 = 0; a0 < nty; a0 += 3)
                for (int c0 = 0; c0 < ntx; c0 += 3) {
                    int at[9];
#pragma unroll
                    for (int u = 0; u < 9; ++u) {
                        const int a = a0 + u / 3, c = c0 + u % 3;
                        at[u] = -1;
                        if (a < nty && c < ntx) {
                            const int b = sl * kp.ntiles + ty[a] * kp.ntx + tx[c];
                            at[u] = kp.tile_start[b] + agg_claim(kp.tile_fill, b);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 9; ++u) {
                        if (at[u] < 0) continue;
                        if (size_t(at[u]) < kp.src_cap) kp.srcsf[at[u]] = r;
                        else atomicOr(kp.status, kStatusCapacity);
                    }
                }
    }
}

// CPT neighbouring x columns per thread (256 / CPT threads for the 16 x 16
// tile): the per-source work of a thread (the loop, the weight loads, the
// zero test) is shared by 8 CPT multiply-adds, issued as 4 CPT packed FP32x2
// FMAs over node pairs. The default is 2; the autotuner may choose 1 or 4.
constexpr int kSpreadCptM = 2;

template <int CPT>
__global__ void __launch_bounds__(kTile * kTile / CPT) k_spread_f32(KP kp) {
    constexpr int B = kSpreadBatchM;
    constexpr int NT = kTile * kTile / CPT, XG = kTile / CPT;
    // x-weight rows padded to a multiple of CPT, so that a thread's CPT
    // weights are one vector load
    constexpr int WXS = CPT == 1 ? kTile + 1 : kTile + CPT;
    __shared__ __align__(16) float s_wx[B][WXS];
    __shared__ float s_wy[B][kTile + 1];
    __shared__ __align__(16) float s_wz[B][kWzStride];
    __shared__ int s_over[B];
    const int tid = threadIdx.x, lx = CPT * (tid % XG), ly = tid / XG;
    const int tile = blockIdx.x, txi = tile % kp.ntx, tyi = tile / kp.ntx;
    const int slab = blockIdx.y, js = slab * kSlabM;
    const int gx0 = txi * kTile, gy0 = tyi * kTile;
    const int bk = slab * kp.ntiles + tile;
    const int first = kp.tile_start[bk], total = kp.tile_start[bk + 1] - first;
    const SrcF* src = kp.srcsf + first;
    const float ig2 = kp.f.ig2, s1 = kp.f.s1norm;
    // the slab's nodes where rho_o is stored (it is zero, and never read, at
    // the nodes it cannot reach)
    unsigned onm = 0xffu;
    if (kp.node_mask) {
        onm = 0u;
        for (int j = 0; j < kSlabM && js + j < kp.nz; ++j) onm |= unsigned(kp.node_mask[js + j] & 1) << j;
    }
    // accumulators as node pairs (j, j + 1): one packed FP32x2 FMA per pair
    float2 ai[CPT][kSlabM / 2], ao[CPT][kSlabM / 2];
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int j = 0; j < kSlabM / 2; ++j) ai[c][j] = ao[c][j] = make_float2(0.f, 0.f);
    for (int base = 0; base < total; base += B) {
        const int nb = min(B, total - base);
        // weight tables: entry b < B of the loop fills source b's x and z
        // weights (times the strength), entry B + b its y weights
        for (int b = tid; b < 2 * B; b += NT) {
            const int rb = b % B;
            if (rb >= nb) continue;
            const SrcF r = src[base + rb];
            if (b < B) {
                const int sx = r.pack & 63;
                int i = wrap_index(gx0 - r.xlo, kp.nx);
                for (int l = 0; l < kTile; ++l) {
                    float w = 0.f;
                    if (i < sx) {
                        const float d = r.d0x + float(i) * kp.f.hx;
                        w = s1 * expf(-d * d * ig2);
                    }
                    s_wx[rb][l] = w;
                    if (++i >= kp.nx) i -= kp.nx;
                }
                const int j0 = (r.pack >> 12) & 511, j1 = (r.pack >> 21) & 511;
                for (int jj = 0; jj < kSlabM; ++jj) {
                    const int j = js + jj;
                    float w = 0.f;
                    if (j >= j0 && j <= j1) {
                        const float d = (kp.zn32[j] - r.zhi) + (kp.znlo32[j] - r.zlo);
                        w = r.q * (s1 * expf(-d * d * ig2));
                    }
                    s_wz[rb][jj] = w;
                }
                s_over[rb] = int((r.pack >> 30) & 1u);
            } else {
                const int sy = (r.pack >> 6) & 63;
                int i = wrap_index(gy0 - r.ylo, kp.ny);
                for (int l = 0; l < kTile; ++l) {
                    float w = 0.f;
                    if (i < sy) {
                        const float d = r.d0y + float(i) * kp.f.hy;
                        w = s1 * expf(-d * d * ig2);
                    }
                    s_wy[rb][l] = w;
                    if (++i >= kp.ny) i -= kp.ny;
                }
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int b = 0; b < nb; ++b) {
            const float wy = s_wy[b][ly];
            if (wy != 0.f) {
                float wxv[CPT];
                if constexpr (CPT == 4) {
                    const float4 t = *reinterpret_cast<const float4*>(&s_wx[b][lx]);
                    wxv[0] = t.x; wxv[1] = t.y; wxv[2] = t.z; wxv[3] = t.w;
                } else if constexpr (CPT == 2) {
                    const float2 t = *reinterpret_cast<const float2*>(&s_wx[b][lx]);
                    wxv[0] = t.x; wxv[1] = t.y;
                } else {
                    wxv[0] = s_wx[b][lx];
                }
                float2 w[CPT];
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    const float v = wxv[c] * wy;
                    w[c] = make_float2(v, v);
                }
                const float4 z0 = *reinterpret_cast<const float4*>(&s_wz[b][0]);
                const float4 z1 = *reinterpret_cast<const float4*>(&s_wz[b][4]);
                const float2 wz[4] = {make_float2(z0.x, z0.y), make_float2(z0.z, z0.w), make_float2(z1.x, z1.y),
                                      make_float2(z1.z, z1.w)};
#pragma unroll
                for (int j = 0; j < kSlabM / 2; ++j)
#pragma unroll
                    for (int c = 0; c < CPT; ++c) ai[c][j] = __ffma2_rn(w[c], wz[j], ai[c][j]);
                if (s_over[b]) {
#pragma unroll
                    for (int j = 0; j < kSlabM / 2; ++j)
#pragma unroll
                        for (int c = 0; c < CPT; ++c) ao[c][j] = __ffma2_rn(w[c], wz[j], ao[c][j]);
                }
            }
        }
        __syncthreads();
    }
    const int gx = gx0 + lx, gy = gy0 + ly;
    if (gy < kp.ny) {
        float* rho = static_cast<float*>(kp.rho);
        const size_t G = size_t(kp.nz) * kp.ny * kp.nx;
#pragma unroll
        for (int j = 0; j < kSlabM; ++j) {
            if (js + j < kp.nz) {
                const size_t g = (size_t(js + j) * kp.ny + gy) * kp.nx + gx;
                const bool on = (onm >> j) & 1u;   // rho_o is zero (and unread) elsewhere
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    if (gx + c < kp.nx) {
                        rho[g + c] = j & 1 ? ai[c][j / 2].y : ai[c][j / 2].x;
                        if (on) rho[G + g + c] = j & 1 ? ao[c][j / 2].y : ao[c][j / 2].x;
                    }
                }
            }
        }
    }
}

template <class R> __device__ __forceinline__ const typename Prec<R>::C* twx_of(const KP& kp);
template <> __device__ __forceinline__ const double2* twx_of<double>(const KP& kp) { return kp.twx; }
template <> __device__ __forceinline__ const float2* twx_of<float>(const KP& kp) { return kp.twx32; }
template <class R> __device__ __forceinline__ const typename Prec<R>::C* twy_of(const KP& kp);
template <> __device__ __forceinline__ const double2* twy_of<double>(const KP& kp) { return kp.twy; }
template <> __device__ __forceinline__ const float2* twy_of<float>(const KP& kp) { return kp.twy32; }

// ---------------------------------------------------------------------------
// xy FFT, forward: rows along x (two real rows packed into one complex FFT),
// then columns along y, for both densities
// ---------------------------------------------------------------------------
// Rows of the pairs p0 .. p0 + P - 1 of a forward x transform (two rows
// each, P <= 64) that are rho_o at nodes it cannot reach: bit q of a (b)
// for the first (second) row of pair q. Those rows are never written, so
// they are read as zero (a pair can straddle two planes when ny is odd);
// all is set when no pair of the block needs a transform.
struct FftxZero {
    unsigned long long a, b;
    bool all;
};
__device__ __forceinline__ FftxZero fftx_zero_rows(const KP& kp, int p0, int P, int npairs) {
    FftxZero z{0ull, 0ull, false};
    if (!kp.node_mask) return z;
    bool all = true;
    for (int q = 0; q < P; ++q) {
        const int pr = p0 + q;
        if (pr >= npairs) continue;
        const bool za = o_row_zero(kp, 2 * pr), zb = o_row_zero(kp, 2 * pr + 1);
        if (za) z.a |= 1ull << q;
        if (zb) z.b |= 1ull << q;
        all = all && za && zb;
    }
    z.all = all;
    return z;
}
// plane (of the 2 nz planes of both densities) of rho_o at a node it cannot reach
__device__ __forceinline__ bool fft_plane_skip(const KP& kp, int plane) {
    return kp.node_mask && plane >= kp.nz && !(kp.node_mask[plane - kp.nz] & 1);
}

template <class R>
__global__ void k_fftx_fwd(KP kp, int P) {
    using C = typename Prec<R>::C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int n = kp.nx, nxh = kp.nxh;
    C* tw = sm;
    C* A = tw + n;
    C* B = A + P * n;
    const C* twg = twx_of<R>(kp);
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const R* rho = static_cast<const R*>(kp.rho);
    C* spec = static_cast<C*>(kp.spec);
    const int npairs = kp.nz * kp.ny;           // 2 nz ny rows
    const int p0 = blockIdx.x * P;
    const FftxZero zr = fftx_zero_rows(kp, p0, P, npairs);
    if (zr.all) return;
    const unsigned long long skip = zr.a & zr.b;
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t / n, x = t - p * n, pr = p0 + p;
        C v;
        v.x = R(0);
        v.y = R(0);
        if (pr < npairs) {
            const size_t r0 = 2 * size_t(pr);
            if (!((zr.a >> p) & 1ull)) v.x = rho[r0 * n + x];
            if (!((zr.b >> p) & 1ull)) v.y = rho[(r0 + 1) * n + x];
        }
        A[p * n + x] = v;
    }
    __syncthreads();
    const C* Rr = block_fft(A, B, tw, n, P, kp.radx, kp.nradx, -1);
    for (int t = threadIdx.x; t < P * nxh; t += blockDim.x) {
        const int p = t / nxh, k = t - p * nxh, pr = p0 + p;
        if (pr >= npairs || ((skip >> p) & 1ull)) continue;
        const C Z = Rr[p * n + k];
        const C Zm = cconj(Rr[p * n + (n - k) % n]);
        const C sum = cadd(Z, Zm), d = csub(Z, Zm);
        const size_t r0 = 2 * size_t(pr);
        spec[r0 * nxh + k] = cscale(sum, R(0.5));
        C b;
        b.x = R(0.5) * d.y;
        b.y = R(-0.5) * d.x;
        spec[(r0 + 1) * nxh + k] = b;
    }
}

template <class R>
__global__ void k_ffty_fwd(KP kp, int TK) {
    using C = typename Prec<R>::C;
    extern __shared__ __align__(16) unsigned char smraw[];
    if (fft_plane_skip(kp, blockIdx.y)) return;
    C* sm = reinterpret_cast<C*>(smraw);
    const int n = kp.ny, nxh = kp.nxh;
    C* tw = sm;
    C* A = tw + n;
    C* B = A + TK * n;
    const C* twg = twy_of<R>(kp);
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    C* base = static_cast<C*>(kp.spec) + size_t(blockIdx.y) * n * nxh;
    const int k0 = blockIdx.x * TK;
    for (int t = threadIdx.x; t < TK * n; t += blockDim.x) {
        const int y = t / TK, c = t - y * TK, kx = k0 + c;
        C v;
        v.x = R(0);
        v.y = R(0);
        if (kx < nxh) v = base[size_t(y) * nxh + kx];
        A[c * n + y] = v;
    }
    __syncthreads();
    const C* Rr = block_fft(A, B, tw, n, TK, kp.rady, kp.nrady, -1);
    for (int t = threadIdx.x; t < TK * n; t += blockDim.x) {
        const int y = t / TK, c = t - y * TK, kx = k0 + c;
        if (kx < nxh) base[size_t(y) * nxh + kx] = Rr[c * n + y];
    }
}

// ---------------------------------------------------------------------------
// xy FFT for power-of-two nx, ny (32..4096): the same four transforms with
// the register radix-16 routine. Rows: P sequences per block; columns: TK
// neighbouring kx columns per block (neighbouring threads on neighbouring
// columns, so every row segment is read and written whole).
// ---------------------------------------------------------------------------
template <class R, int L>
__global__ void k_fftx_fwd_p2(KP kp, int P, int) {
    using C = typename Prec<R>::C;
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int logn = L, n = 1 << L, nxh = n / 2 + 1, np = n + (n >> 4);
    C* buf = reinterpret_cast<C*>(smraw);
    const C* tw = twx_of<R>(kp);
    const R* rho = static_cast<const R*>(kp.rho);
    C* spec = static_cast<C*>(kp.spec);
    const int npairs = kp.nz * kp.ny;
    const int p0 = blockIdx.x * P;
    const FftxZero zr = fftx_zero_rows(kp, p0, P, npairs);
    if (zr.all) return;
    const unsigned long long skip = zr.a & zr.b;
    auto load = [&](int q, int i) {
        C v;
        v.x = R(0);
        v.y = R(0);
        if (p0 + q < npairs) {
            const size_t r0 = 2 * size_t(p0 + q);
            if (!((zr.a >> q) & 1ull)) v.x = rho[r0 * n + i];
            if (!((zr.b >> q) & 1ull)) v.y = rho[(r0 + 1) * n + i];
        }
        return v;
    };
    auto store = [&](int q, int i, C v) { buf[q * np + pad16(i)] = v; };
    fft_pow2<false>(buf, tw, n, logn, P, -1, load, store);
    __syncthreads();
    for (int t = threadIdx.x; t < P * nxh; t += blockDim.x) {
        const int p = t / nxh, k = t - p * nxh, pr = p0 + p;
        if (pr >= npairs || ((skip >> p) & 1ull)) continue;
        const C Z = buf[p * np + pad16(k)];
        const C Zm = cconj(buf[p * np + pad16((n - k) & (n - 1))]);
        const C sum = cadd(Z, Zm), d = csub(Z, Zm);
        const size_t r0 = 2 * size_t(pr);
        spec[r0 * nxh + k] = cscale(sum, R(0.5));
        C b;
        b.x = R(0.5) * d.y;
        b.y = R(-0.5) * d.x;
        spec[(r0 + 1) * nxh + k] = b;
    }
}

template <class R, int L>
__global__ void k_ffty_fwd_p2(KP kp, int TK, int) {
    using C = typename Prec<R>::C;
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int logn = L, n = 1 << L;
    const int nxh = kp.nxh;
    if (fft_plane_skip(kp, blockIdx.y)) return;
    C* tw = reinterpret_cast<C*>(smraw);
    C* buf = tw + n;
    C* base = static_cast<C*>(kp.spec) + size_t(blockIdx.y) * n * nxh;
    const int k0 = blockIdx.x * TK;
    auto load = [&](int q, int i) {
        C v;
        v.x = R(0);
        v.y = R(0);
        if (k0 + q < nxh) v = base[size_t(i) * nxh + k0 + q];
        return v;
    };
    auto store = [&](int q, int i, C v) {
        if (k0 + q < nxh) base[size_t(i) * nxh + k0 + q] = v;
    };
    fft_pow2<true>(buf, tw, n, logn, TK, -1, load, store, tw, twy_of<R>(kp));
}

// one of the three inverse column transforms: F = 0: -i k_y psi (psi -> specB),
// F = 1: psi (in place), F = 2: dpsi/dz (in place)
template <int F, class R, int L>
__device__ __forceinline__ void ffty_inv_field(const KP& kp, typename Prec<R>::C* buf, typename Prec<R>::C* tw,
                                               int TK, bool fill) {
    using C = typename Prec<R>::C;
    constexpr int logn = L, n = 1 << L;
    const int nxh = kp.nxh;
    const size_t plane = size_t(n) * nxh;
    C* src = static_cast<C*>(kp.spec) + size_t((F == 2 ? kp.nz : 0) + blockIdx.y) * plane;
    C* dst = F == 0 ? static_cast<C*>(kp.specB) + size_t(blockIdx.y) * plane : src;
    const R kys = R(kTwoPi / kp.Ly);
    const int k0 = blockIdx.x * TK;
    auto load = [&](int c, int i) {
        C v;
        v.x = R(0);
        v.y = R(0);
        if (k0 + c >= nxh) return v;
        const C ps = src[size_t(i) * nxh + k0 + c];
        if constexpr (F != 0) return ps;
        const int my = i < (n + 1) / 2 ? i : i - n;
        const R ky = (i == n / 2) ? R(0) : (sizeof(R) == sizeof(double) ? R(kTwoPi * my / kp.Ly) : kys * R(my));
        v.x = ky * ps.y;
        v.y = -ky * ps.x;
        return v;
    };
    auto store = [&](int c, int i, C v) {
        if (k0 + c < nxh) dst[size_t(i) * nxh + k0 + c] = v;
    };
    fft_pow2<true>(buf, tw, n, logn, TK, +1, load, store, fill ? tw : nullptr, twy_of<R>(kp));
}

template <class R, int L>
__global__ void __launch_bounds__(512, sizeof(R) == sizeof(float) ? 2 : 1) k_ffty_inv_p2(KP kp, int TK, int) {
    using C = typename Prec<R>::C;
    extern __shared__ __align__(16) unsigned char smraw[];
    if (kp.node_mask && !(kp.node_mask[blockIdx.y] & 2)) return;   // a plane the interpolation never reads
    C* tw = reinterpret_cast<C*>(smraw);
    C* buf = tw + (1 << L);
    // -i k_y psi first: it reads psi before the psi transform overwrites it
    // (the first transform also copies the twiddle table)
    ffty_inv_field<0, R, L>(kp, buf, tw, TK, true);
    __syncthreads();
    ffty_inv_field<1, R, L>(kp, buf, tw, TK, false);
    __syncthreads();
    ffty_inv_field<2, R, L>(kp, buf, tw, TK, false);
}

template <class R, int L>
__global__ void k_fftx_inv_p2(KP kp, int P, int) {
    using C = typename Prec<R>::C;
    using V4 = typename Prec<R>::V4;
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int logn = L, n = 1 << L, nxh = n / 2 + 1, n16 = n >> 4;
    C* buf = reinterpret_cast<C*>(smraw);
    const C* tw = twx_of<R>(kp);
    const C* spec = static_cast<const C*>(kp.spec);
    const C* specB = static_cast<const C*>(kp.specB);
    V4* fields = static_cast<V4*>(kp.fields);
    const int nrows = kp.nz * kp.ny;
    const size_t S = size_t(nrows) * nxh;
    const R kxs = R(kTwoPi / kp.Lx);
    const int r0 = blockIdx.x * P;
    // rows past the grid or at nodes the interpolation never reads
    const unsigned long long skip = f_rows_skip(kp, r0, P, nrows);
    if (skip == (P >= 64 ? ~0ull : (1ull << P) - 1ull)) return;
    // sequence q = 2 p + w: row r0 + p; w = 0 packs (phi, E_x), w = 1 (E_y, E_z)
    auto load = [&](int q, int k) {
        const int p = q >> 1, w = q & 1, row = r0 + p;
        C z;
        z.x = R(0);
        z.y = R(0);
        if ((skip >> p) & 1ull) return z;
        const bool hi = k >= nxh;
        const int kk = hi ? n - k : k;
        const bool edge = kk == 0 || kk == n / 2;
        const size_t g = size_t(row) * nxh + kk;
        // the two lanes of a row pair take the same steps (no divergence):
        // w = 0: a = psi, s = -i k_x psi, z = phi + i E_x;
        // w = 1: a = -i k_y psi, s = -dpsi/dz, z = E_y + i E_z
        C a = (w ? specB : spec)[g];
        C c;
        c.x = R(0);
        c.y = R(0);
        if (w) c = spec[S + g];
        if (edge) { a.y = R(0); c.y = R(0); }
        const R kxd = edge ? R(0) : (sizeof(R) == sizeof(double) ? R(kTwoPi * kk / kp.Lx) : kxs * R(kk));
        C sv;
        sv.x = w ? -c.x : kxd * a.y;
        sv.y = w ? -c.y : -kxd * a.x;
        if (hi) { a = cconj(a); sv = cconj(sv); }
        z.x = a.x - sv.y;
        z.y = a.y + sv.x;
        return z;
    };
    // the two sequences of a row sit on neighbouring lanes (w = lane parity)
    // and hold the same outputs x = j + g n16: the w = 0 lane stores the even
    // g, the w = 1 lane the odd g, each taking the other half from its
    // partner by a shuffle, so the outputs need no second pass through
    // shared memory
    const R s = R(kp.inv_nxny);
    const int wlanes = min(32, int(blockDim.x) - (int(threadIdx.x) & ~31));
    const unsigned wmask = wlanes == 32 ? 0xffffffffu : (1u << wlanes) - 1u;
    auto store = [&](int q, int j, bool act, C(&v)[16]) {
        const int p = q >> 1, w = q & 1;
        const bool keep = act && !((skip >> p) & 1ull);
        V4* out = fields + size_t(r0 + p) * n + j;
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const C send = w ? v[2 * h] : v[2 * h + 1];
            C recv;
            recv.x = __shfl_xor_sync(wmask, send.x, 1);
            recv.y = __shfl_xor_sync(wmask, send.y, 1);
            const C u = w ? recv : v[2 * h], e = w ? v[2 * h + 1] : recv;
            if (keep) out[(2 * h + w) * n16] = Prec<R>::v4(u.x * s, u.y * s, e.x * s, e.y * s);
        }
    };
    fft_pow2<false, false, true>(buf, tw, n, logn, 2 * P, +1, load, store);
}

// The power-of-two kernels are compiled for each n = 2^L (32 <= n <= 4096),
// so that their index arithmetic folds to constants. which: 0 x forward,
// 1 y forward, 2 y inverse, 3 x inverse; nullptr for other sizes.
using FftP2Kernel = void (*)(KP, int, int);
template <class R, int L>
FftP2Kernel fft_p2_at(int which) {
    return which == 0 ? k_fftx_fwd_p2<R, L> : which == 1 ? k_ffty_fwd_p2<R, L>
         : which == 2 ? k_ffty_inv_p2<R, L> : k_fftx_inv_p2<R, L>;
}
template <class R>
FftP2Kernel fft_p2(int which, int logn) {
    switch (logn) {
        case 5: return fft_p2_at<R, 5>(which);
        case 6: return fft_p2_at<R, 6>(which);
        case 7: return fft_p2_at<R, 7>(which);
        case 8: return fft_p2_at<R, 8>(which);
        case 9: return fft_p2_at<R, 9>(which);
        case 10: return fft_p2_at<R, 10>(which);
        case 11: return fft_p2_at<R, 11>(which);
        case 12: return fft_p2_at<R, 12>(which);
        default: return nullptr;
    }
}

// ---------------------------------------------------------------------------
// per-mode column work: z Chebyshev transform, the Appendix-A BVP for both
// densities, mismatches and correction (Sec. 5.2.2 step 4), the k = 0 slope
// (step 5), the gauge partial sum, and the values of psi_i and dpsi_i/dz at
// the nodes (step 6); written in place over the two spectra
// ---------------------------------------------------------------------------
template <int CB>
__device__ __forceinline__ void column_body(const KP& kp, const int bid) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = kp.nz;
    const int M = kp.ny * kp.nxh;
    double2* Vi = reinterpret_cast<double2*>(smraw);   // values, then y' (field i)
    double2* Vo = Vi + CB * N;                         // values, then y' (field o)
    double2* Ci = Vo + CB * N;                         // coefficients -> y'' -> y
    double2* Co = Ci + CB * N;
    double* cpv = reinterpret_cast<double*>(Co + CB * N);   // Thomas c'
    double* xe = cpv + CB * N;                               // K^2 A^{-1} e0 (even) / e1 (odd)
    __shared__ double s_k[CB], s_K[CB], s_mult[CB], s_den[CB], s_ekH[CB], s_gauge[CB];
    __shared__ int s_valid[CB], s_corr[CB];
    __shared__ double2 s_c[2][CB], s_d[2][CB], s_P[CB], s_Q[CB];
    __shared__ double s_Ai;
    const int tid = threadIdx.x, bs = blockDim.x;
    const int col0 = bid * CB;
    const double Hbar = kp.Hbar;
    double2* const spd = static_cast<double2*>(kp.spec);

    if (tid < CB) {
        const int c = tid, col = col0 + c;
        const int iy = col / kp.nxh, ix = col - iy * kp.nxh;
        const int my = iy < (kp.ny + 1) / 2 ? iy : iy - kp.ny;
        const double kx = kTwoPi * ix / kp.Lx, ky = kTwoPi * my / kp.Ly;
        const double k = sqrt(kx * kx + ky * ky);
        s_valid[c] = col < M;
        s_k[c] = k;
        s_K[c] = 0.5 * k * Hbar;
        s_mult[c] = (ix == 0 || (kp.nx % 2 == 0 && ix == kp.nx / 2)) ? 1.0 : 2.0;
        s_corr[c] = (col < M) && k > 0.0 && k <= kp.kmax;
        s_gauge[c] = 0.0;
    }
    if (tid == 0) s_Ai = 0.0;
    for (int t = tid; t < N * CB; t += bs) {
        const int j = t / CB, c = t - j * CB, col = col0 + c;
        double2 vi = make_double2(0.0, 0.0), vo = vi;
        if (col < M) {
            vi = spd[size_t(j) * M + col];
            vo = spd[size_t(N + j) * M + col];
        }
        Vi[c * N + j] = vi;
        Vo[c * N + j] = vo;
    }
    __syncthreads();

    // coefficients f_n = sum_j cf[n][j] v_j, then F = -(Hbar/2)^2 f / eps,
    // split by the node symmetry: V[a] <- v_a + v_{m-a}, V[m-a] <- v_a - v_{m-a}
    const int m = N - 1, JE = (N + 1) / 2, JO = N / 2;
    for (int t = tid; t < 2 * CB * JE; t += bs) {
        const int f = t / (CB * JE), r = t - f * CB * JE, c = r / JE, a = r - c * JE;
        if (a < m - a) {
            double2* V = (f ? Vo : Vi) + c * N;
            const double2 va = V[a], vb = V[m - a];
            V[a] = cadd(va, vb);
            V[m - a] = csub(va, vb);
        }
    }
    __syncthreads();
    const double scale = -(0.5 * Hbar) * (0.5 * Hbar) / kp.eps;
    // thread (c, q): output row q of both densities; q < JE even n = 2q from
    // S_a = V[a], q >= JE odd n from D_a = V[m - a]; lanes run over q so the
    // table loads are contiguous and the V loads are broadcasts
    for (int t = tid; t < CB * N; t += bs) {
        const int c = t / N, q = t - c * N;
        const bool odd = q >= JE;
        const int na = odd ? JO : JE;
        const double2* vi = Vi + c * N;
        const double2* vo = Vo + c * N;
        double ix = 0.0, iy = 0.0, ox = 0.0, oy = 0.0;
        for (int a = 0; a < na; ++a) {
            const double w = kp.cft[size_t(a) * N + q];
            const int ia = odd ? m - a : a;
            const double2 u = vi[ia], v = vo[ia];
            ix = fma(w, u.x, ix);
            iy = fma(w, u.y, iy);
            ox = fma(w, v.x, ox);
            oy = fma(w, v.y, oy);
        }
        const int n = odd ? 2 * (q - JE) + 1 : 2 * q;
        Ci[c * N + n] = make_double2(ix * scale, iy * scale);
        Co[c * N + n] = make_double2(ox * scale, oy * scale);
    }
    __syncthreads();

    // Appendix A: A y'' = F + K^2 (c e0 + d e1), A = I - K^2 J^2 splits into the
    // even and odd index chains, each tridiagonal (Thomas algorithm).
    if (tid < 2 * CB) {
        const int c = tid >> 1, ch = tid & 1;
        const double K2 = s_K[c] * s_K[c];
        double2* Fi = Ci + c * N;
        double2* Fo = Co + c * N;
        double* cq = cpv + c * N;
        double* xc = xe + c * N;
        int prev = -1;
        for (int n = ch; n < N; n += 2) {
            const double an = n >= 2 ? -K2 * kp.j2l[n] : 0.0;
            const double bn = 1.0 - K2 * kp.j2d[n];
            const double cn = n + 2 < N ? -K2 * kp.j2u[n] : 0.0;
            double m = bn, rn = (n == ch) ? K2 : 0.0;
            double2 fi = Fi[n], fo = Fo[n];
            if (prev >= 0) {
                m -= an * cq[prev];
                fi = csub(fi, cscale(Fi[prev], an));
                fo = csub(fo, cscale(Fo[prev], an));
                rn -= an * xc[prev];
            }
            const double inv = 1.0 / m;
            cq[n] = cn * inv;
            Fi[n] = cscale(fi, inv);
            Fo[n] = cscale(fo, inv);
            xc[n] = rn * inv;
            prev = n;
        }
        for (int n = prev - 2; n >= ch; n -= 2) {
            Fi[n] = csub(Fi[n], cscale(Fi[n + 2], cq[n]));
            Fo[n] = csub(Fo[n], cscale(Fo[n + 2], cq[n]));
            xc[n] -= cq[n] * xc[n + 2];
        }
    }
    __syncthreads();

    // 2x2 Schur complement for the integration constants (y_0, y'_0) = (c, d)
    // from the two boundary rows (Eq. (BCs); Eq. (BCs0) for k = 0); warp w
    // handles column w, lanes split the sums over n
    {
        const int c = tid >> 5, lane = tid & 31;
        const double K = s_K[c];
        const double2* Xi = Ci + c * N;
        const double2* Xo = Co + c * N;
        const double* xc = xe + c * N;
        double acc[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int n = lane; n < N; n += 32) {
            const double gtn = K > 0.0 ? kp.u1[n] + K * kp.u2[n] : kp.u2[n];
            const double gbn = K > 0.0 ? kp.v1[n] - K * kp.v2[n] : kp.v2[n];
            acc[0] = fma(gtn, Xi[n].x, acc[0]); acc[1] = fma(gtn, Xi[n].y, acc[1]);
            acc[2] = fma(gbn, Xi[n].x, acc[2]); acc[3] = fma(gbn, Xi[n].y, acc[3]);
            acc[4] = fma(gtn, Xo[n].x, acc[4]); acc[5] = fma(gtn, Xo[n].y, acc[5]);
            acc[6] = fma(gbn, Xo[n].x, acc[6]); acc[7] = fma(gbn, Xo[n].y, acc[7]);
            if (n & 1) { acc[9] = fma(gtn, xc[n], acc[9]); acc[11] = fma(gbn, xc[n], acc[11]); }
            else { acc[8] = fma(gtn, xc[n], acc[8]); acc[10] = fma(gbn, xc[n], acc[10]); }
        }
        {   // the 12 sums (lane 4 v: value v < 8, lane 8 v: value 8 + v), gathered
            const double r8 = warp_sum_multi<8>(acc), r4 = warp_sum_multi<4>(acc + 8);
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = __shfl_sync(0xffffffffu, r8, 4 * i);
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[8 + i] = __shfl_sync(0xffffffffu, r4, 8 * i);
        }
        if (lane < 2) {
            const int f = lane;
            const double2 sFt = f ? make_double2(acc[4], acc[5]) : make_double2(acc[0], acc[1]);
            const double2 sFb = f ? make_double2(acc[6], acc[7]) : make_double2(acc[2], acc[3]);
            double2 cc, dd;
            if (K > 0.0) {
                const double m11 = K + acc[8], m12 = 1.0 + K + acc[9], m21 = -K + acc[10], m22 = 1.0 + K + acc[11];
                const double idet = 1.0 / (m11 * m22 - m12 * m21);
                cc = cscale(csub(cscale(sFt, m22), cscale(sFb, m12)), -idet);
                dd = cscale(csub(cscale(sFb, m11), cscale(sFt, m21)), -idet);
            } else {
                // sum y_n = c + d + u2.y'' = 0, sum (-1)^n y_n = c - d + v2.y'' = 0
                cc = cscale(cadd(sFt, sFb), -0.5);
                dd = cscale(csub(sFt, sFb), -0.5);
            }
            s_c[f][c] = cc;
            s_d[f][c] = dd;
        }
    }
    __syncthreads();
    // y'' = x_F + c x_c + d x_d
    for (int t = tid; t < 2 * CB * N; t += bs) {
        const int f = t / (CB * N), r = t - f * CB * N, c = r / N, n = r - c * N;
        double2* X = (f ? Co : Ci) + c * N;
        const double2 m = (n & 1) ? s_d[f][c] : s_c[f][c];
        X[n] = cadd(X[n], cscale(m, xe[c * N + n]));
    }
    __syncthreads();
    // y' from y'' (Eq. (ds)), into the value buffers
    for (int t = tid; t < 2 * CB * N; t += bs) {
        const int f = t / (CB * N), r = t - f * CB * N, c = r / N, n = r - c * N;
        const double2* Y = (f ? Co : Ci) + c * N;
        double2 v;
        if (n == 0) v = s_d[f][c];
        else if (n == 1) v = csub(Y[0], cscale(Y[2], 0.5));
        else v = cscale(csub(Y[n - 1], n + 1 < N ? Y[n + 1] : make_double2(0.0, 0.0)), 0.5 / n);
        (f ? Vo : Vi)[c * N + n] = v;
    }
    __syncthreads();
    // y from y' (Eq. (cs)), over y''
    for (int t = tid; t < 2 * CB * N; t += bs) {
        const int f = t / (CB * N), r = t - f * CB * N, c = r / N, n = r - c * N;
        const double2* Y = (f ? Vo : Vi) + c * N;
        double2 v;
        if (n == 0) v = s_c[f][c];
        else if (n == 1) v = csub(Y[0], cscale(Y[2], 0.5));
        else v = cscale(csub(Y[n - 1], n + 1 < N ? Y[n + 1] : make_double2(0.0, 0.0)), 0.5 / n);
        (f ? Co : Ci)[c * N + n] = v;
    }
    __syncthreads();

    // boundary values, mismatches Eq. (mm1)-(mm4), correction coefficients,
    // k = 0 slope, gauge partial sum (warp per column, lanes over n)
    {
        const int c = tid >> 5, lane = tid & 31;
        const double2 *yi = Ci + c * N, *ypi = Vi + c * N, *yo = Co + c * N, *ypo = Vo + c * N;
        double acc[22];
        for (int i = 0; i < 22; ++i) acc[i] = 0.0;
        for (int n = lane; n < N; n += 32) {
            const double a0 = kp.t0[n], aH = kp.tH[n], alt = (n & 1) ? -1.0 : 1.0, wg = kp.wg[n];
            acc[0] = fma(a0, yi[n].x, acc[0]);   acc[1] = fma(a0, yi[n].y, acc[1]);     // psi_i*(0)
            acc[2] = fma(a0, ypi[n].x, acc[2]);  acc[3] = fma(a0, ypi[n].y, acc[3]);    // psi_i*'(0)
            acc[4] = fma(aH, yi[n].x, acc[4]);   acc[5] = fma(aH, yi[n].y, acc[5]);     // psi_i*(H)
            acc[6] = fma(aH, ypi[n].x, acc[6]);  acc[7] = fma(aH, ypi[n].y, acc[7]);    // psi_i*'(H)
            acc[8] = fma(a0, yo[n].x, acc[8]);   acc[9] = fma(a0, yo[n].y, acc[9]);     // psi_o*(0)
            acc[10] = fma(a0, ypo[n].x, acc[10]); acc[11] = fma(a0, ypo[n].y, acc[11]); // psi_o*'(0)
            acc[12] = fma(aH, yo[n].x, acc[12]); acc[13] = fma(aH, yo[n].y, acc[13]);   // psi_o*(H)
            acc[14] = fma(aH, ypo[n].x, acc[14]); acc[15] = fma(aH, ypo[n].y, acc[15]); // psi_o*'(H)
            acc[16] = fma(alt, ypo[n].x, acc[16]); acc[17] += ypo[n].x;                // psi_o*'(a), (b)
            acc[18] = fma(wg, yi[n].x, acc[18]); acc[19] = fma(wg, yi[n].y, acc[19]);   // gauge sum
        }
        {   // the 20 sums (lane 2 v: value v < 16, lane 8 v: value 16 + v), gathered
            const double r16 = warp_sum_multi<16>(acc), r4 = warp_sum_multi<4>(acc + 16);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = __shfl_sync(0xffffffffu, r16, 2 * i);
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[16 + i] = __shfl_sync(0xffffffffu, r4, 8 * i);
        }
        if (lane == 0 && s_valid[c]) {
            const double dz = 2.0 / Hbar;
            const double2 pi0 = make_double2(acc[0], acc[1]), dpi0 = make_double2(acc[2] * dz, acc[3] * dz);
            const double2 piH = make_double2(acc[4], acc[5]), dpiH = make_double2(acc[6] * dz, acc[7] * dz);
            const double2 po0 = make_double2(acc[8], acc[9]), dpo0 = make_double2(acc[10] * dz, acc[11] * dz);
            const double2 poH = make_double2(acc[12], acc[13]), dpoH = make_double2(acc[14] * dz, acc[15] * dz);
            const double dpoa = acc[16] * dz, dpob = acc[17] * dz;
            const double k = s_k[c];
            double2 corr0 = make_double2(0.0, 0.0);
            if (s_corr[c]) {
                const double2 mpb = csub(pi0, cscale(po0, kp.tb));
                double2 meb = csub(dpi0, cscale(dpo0, kp.rtb));
                const double2 mpt = csub(piH, cscale(poH, kp.tt));
                double2 met = csub(dpiH, cscale(dpoH, kp.rtt));
                if (kp.sigma_on) {   // Eq. (mm2), (mm4): +sigma_b, -sigma_t (over eps)
                    meb = cadd(meb, cscale(kp.sig_hat[col0 + c], 1.0 / kp.eps));
                    met = csub(met, cscale(kp.sig_hat[M + col0 + c], 1.0 / kp.eps));
                }
                const double2 P = csub(cscale(mpb, kp.cb), cscale(meb, kp.db / k));
                const double2 Q = csub(cscale(mpt, -kp.ct), cscale(met, kp.dt / k));
                const double ekH = exp(-k * kp.H);
                const double den = 1.0 - kp.Gb * kp.Gt * ekH * ekH;
                s_P[c] = P;
                s_Q[c] = Q;
                s_ekH[c] = ekH;
                s_den[c] = den;
                corr0 = cscale(cadd(cscale(P, -(1.0 - kp.Gt * ekH * ekH)), cscale(Q, ekH - kp.Gb * ekH)), 1.0 / den);
            }
            if (col0 + c == 0) {
                // Sec. 4.3.4: Eq. (CE), (ai1), (ai2); mean, or the non-metal wall's
                // equation, or equal wall potentials for two metal walls
                double ai1 = kp.rtb * (dpo0.x - dpoa) - dpi0.x;
                double ai2 = kp.rtt * (dpoH.x - dpob) - dpiH.x;
                if (kp.sigma_on) {
                    ai1 -= kp.sig_hat[0].x / kp.eps;
                    ai2 += kp.sig_hat[M].x / kp.eps;
                }
                double Ai;
                if (kp.metal_b && kp.metal_t) Ai = -(piH.x - pi0.x) / kp.H;
                else if (kp.metal_b) Ai = ai2;
                else if (kp.metal_t) Ai = ai1;
                else Ai = 0.5 * (ai1 + ai2);
                s_Ai = Ai;
                kp.scal[1] = Ai;
                if (kp.sigma_on) {   // k = 0 far potential at the walls, gamma^{1/2}-averaged in z
                    double f0 = 0.0, fH = 0.0;
                    for (int n = 0; n < N; ++n) {
                        f0 = fma(kp.wg[n], yi[n].x, f0);
                        fH = fma(kp.wgH[n], yi[n].x, fH);
                    }
                    kp.scal[7] = f0;
                    kp.scal[8] = fH + Ai * kp.H;
                }
            }
            const double damp = exp(-0.5 * kp.sigma2 * k * k);
            s_gauge[c] = s_mult[c] * (damp * acc[18] + corr0.x);
        }
    }
    __syncthreads();

    // node values of psi_i and dpsi_i/dz (+ correction, + A_i z for k = 0):
    // nodes a and m-a from the even (E) and odd (O) coefficient sums, E +/- O
    const double Ai = s_Ai;
    for (int t = tid; t < JE * CB; t += bs) {
        const int c = t / JE, a = t - c * JE, col = col0 + c;
        if (col >= M) continue;
        const double2* yi = Ci + c * N;
        const double2* ypi = Vi + c * N;
        double ex = 0, ey = 0, dex = 0, dey = 0, ox = 0, oy = 0, dox = 0, doy = 0;
        for (int r = 0; r < JE; ++r) {
            const double w = kp.tie[size_t(r) * JE + a];
            ex = fma(w, yi[2 * r].x, ex);
            ey = fma(w, yi[2 * r].y, ey);
            dex = fma(w, ypi[2 * r].x, dex);
            dey = fma(w, ypi[2 * r].y, dey);
        }
        for (int r = 0; r < JO; ++r) {
            const double w = kp.tio[size_t(r) * JE + a];
            ox = fma(w, yi[2 * r + 1].x, ox);
            oy = fma(w, yi[2 * r + 1].y, oy);
            dox = fma(w, ypi[2 * r + 1].x, dox);
            doy = fma(w, ypi[2 * r + 1].y, doy);
        }
        const double sz = 2.0 / Hbar;
        for (int side = 0; side < 2; ++side) {
            const int j = side ? m - a : a;
            if (side && j == a) break;
            const double sg = side ? -1.0 : 1.0;
            double2 ps = make_double2(ex + sg * ox, ey + sg * oy);
            double2 dps = make_double2((dex + sg * dox) * sz, (dey + sg * doy) * sz);
            const double z = kp.zn[j];
            if (s_corr[c] && z >= -kp.HE && z <= kp.H + kp.HE) {
                const double k = s_k[c], ekH = s_ekH[c], iden = 1.0 / s_den[c];
                const double e1 = exp(-k * z), e3 = exp(k * (z - kp.H));
                const double e2 = e3 * ekH, e4 = e1 * ekH;
                const double2 P = s_P[c], Q = s_Q[c];
                const double2 val = cscale(cadd(cscale(P, -(e1 - kp.Gt * e2)), cscale(Q, e3 - kp.Gb * e4)), iden);
                const double2 der = cscale(cadd(cscale(P, e1 + kp.Gt * e2), cscale(Q, e3 + kp.Gb * e4)), k * iden);
                ps = cadd(ps, val);
                dps = cadd(dps, der);
            }
            if (col == 0) {
                ps.x += Ai * z;
                dps.x += Ai;
            }
            spd[size_t(j) * M + col] = ps;
            spd[size_t(N + j) * M + col] = dps;
        }
    }
    const double g = block_sum(tid < CB ? s_gauge[tid] : 0.0);
    if (tid == 0) kp.part_gauge_far[bid] = g;
}
template <int CB>
__global__ void __launch_bounds__(32 * CB) k_column(KP kp) { column_body<CB>(kp, blockIdx.x); }
__global__ void __launch_bounds__(kColThreads) k_column_batch(const __grid_constant__ ColBatch b) {
    const int s = batch_system(b.starts, b.nsys, blockIdx.x);
    column_body<kColBlock>(b.kp[s], blockIdx.x - b.starts[s]);
}

// ---------------------------------------------------------------------------
// The k = 0 column of the mixed-precision solve, in double, in one block:
// the z transform of the two densities' plane sums (the xy transform's DC
// bins), the Appendix-A BVP at k = 0 (A = I, so y'' = F, and the two
// Dirichlet rows Eq. (BCs0) give y_0 and y'_0), the slope A_i of Sec. 4.3.4
// (Eq. (CE), (ai1), (ai2)), this column's part of the gauge sum and, with
// wall charges, the k = 0 far potential at the walls. It runs after the xy
// transforms, before any z transform, and leaves the coefficients of psi_i
// and dpsi_i/dz (before the factor 2/Hbar) in kp.zcol for k_column_mixed.
// ---------------------------------------------------------------------------
constexpr int kZeroThreads = 256;

// Sums over the block of V values per thread, in a fixed order; every thread
// must call it, and out (shared) holds the V sums on return.
template <int V>
__device__ void block_sums(const double (&v)[V], double* out) {
    __shared__ double red[V][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const double s = warp_sum(v[i]);
        if (lane == 0) red[i][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < V) {
        double s = 0.0;
        for (int k = 0; k < nw; ++k) s += red[threadIdx.x][k];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void column_zero_body(const KP& kp) {
    __shared__ double s_v[2][kMaxNz];   // node values, split into S_a / D_a
    __shared__ double s_y[2][kMaxNz];   // F = y'' (k = 0), then y
    __shared__ double s_p[2][kMaxNz];   // y'
    __shared__ double s_sum[16];
    const int N = kp.nz, M = kp.ny * kp.nxh, tid = threadIdx.x, bs = blockDim.x;
    const float2* sp = static_cast<const float2*>(kp.spec);
    // column 0 of both spectra: the plane sums of rho_i, rho_o (real)
    for (int t = tid; t < 2 * N; t += bs)
        s_v[t / N][t % N] = (t >= N && kp.node_mask && !(kp.node_mask[t - N] & 1)) ? 0.0 : double(sp[size_t(t) * M].x);
    __syncthreads();
    const int m = N - 1, JE = (N + 1) / 2, JO = N / 2;
    for (int t = tid; t < 2 * JE; t += bs) {
        const int f = t / JE, a = t - f * JE;
        if (a < m - a) {
            const double va = s_v[f][a], vb = s_v[f][m - a];
            s_v[f][a] = va + vb;
            s_v[f][m - a] = va - vb;
        }
    }
    __syncthreads();
    // coefficients (split forward transform, as in k_column), times
    // -(Hbar/2)^2/eps: the right-hand side F of Eq. (blocksys)
    const double scale = -(0.5 * kp.Hbar) * (0.5 * kp.Hbar) / kp.eps;
    for (int t = tid; t < 2 * N; t += bs) {
        const int f = t / N, q = t - f * N;
        const bool odd = q >= JE;
        const int na = odd ? JO : JE;
        double acc = 0.0;
        for (int a = 0; a < na; ++a) acc = fma(kp.cft[size_t(a) * N + q], s_v[f][odd ? m - a : a], acc);
        s_y[f][odd ? 2 * (q - JE) + 1 : 2 * q] = acc * scale;
    }
    __syncthreads();
    // k = 0 rows: sum y_n = c + d + u2.y'' = 0, sum (-1)^n y_n = c - d + v2.y'' = 0
    {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int n = tid; n < N; n += bs) {
            v[0] = fma(kp.u2[n], s_y[0][n], v[0]);
            v[1] = fma(kp.v2[n], s_y[0][n], v[1]);
            v[2] = fma(kp.u2[n], s_y[1][n], v[2]);
            v[3] = fma(kp.v2[n], s_y[1][n], v[3]);
        }
        block_sums<4>(v, s_sum);
    }
    // y' = J y'' + d e0, then y = J y' + c e0 (entry n of J v is
    // (v_{n-1} - v_{n+1})/(2n), entry 1 is v_0 - v_2/2)
    for (int t = tid; t < 2 * N; t += bs) {
        const int f = t / N, n = t - f * N;
        const double* Y = s_y[f];
        double v;
        if (n == 0) v = -0.5 * (s_sum[2 * f] - s_sum[2 * f + 1]);
        else if (n == 1) v = Y[0] - 0.5 * (N > 2 ? Y[2] : 0.0);
        else v = (Y[n - 1] - (n + 1 < N ? Y[n + 1] : 0.0)) * (0.5 / n);
        s_p[f][n] = v;
    }
    __syncthreads();
    for (int t = tid; t < 2 * N; t += bs) {
        const int f = t / N, n = t - f * N;
        const double* Y = s_p[f];
        double v;
        if (n == 0) v = -0.5 * (s_sum[2 * f] + s_sum[2 * f + 1]);
        else if (n == 1) v = Y[0] - 0.5 * (N > 2 ? Y[2] : 0.0);
        else v = (Y[n - 1] - (n + 1 < N ? Y[n + 1] : 0.0)) * (0.5 / n);
        s_y[f][n] = v;    // y'' of this n is no longer read: n - 1 and n + 1 of y' are
    }
    __syncthreads();
    // boundary values (Sec. 4.3.4 needs psi_i*, d psi_i*/dz at z = 0, H and
    // d psi_o*/dz at z = 0, H, a, b), the gauge sum, the wall potentials
    {
        double v[11];
#pragma unroll
        for (int i = 0; i < 11; ++i) v[i] = 0.0;
        for (int n = tid; n < N; n += bs) {
            const double a0 = kp.t0[n], aH = kp.tH[n], alt = (n & 1) ? -1.0 : 1.0;
            const double yi = s_y[0][n], ypi = s_p[0][n], ypo = s_p[1][n];
            v[0] = fma(a0, yi, v[0]);
            v[1] = fma(aH, yi, v[1]);
            v[2] = fma(a0, ypi, v[2]);
            v[3] = fma(aH, ypi, v[3]);
            v[4] = fma(a0, ypo, v[4]);
            v[5] = fma(aH, ypo, v[5]);
            v[6] = fma(alt, ypo, v[6]);
            v[7] += ypo;
            v[8] = fma(kp.wg[n], yi, v[8]);
            if (kp.sigma_on) v[9] = fma(kp.wgH[n], yi, v[9]);
        }
        block_sums<11>(v, s_sum);
    }
    for (int t = tid; t < 2 * N; t += bs) kp.zcol[t] = t < N ? s_y[0][t] : s_p[0][t - N];
    if (tid == 0) {
        const double dz = 2.0 / kp.Hbar;
        const double pi0 = s_sum[0], piH = s_sum[1];
        const double dpi0 = s_sum[2] * dz, dpiH = s_sum[3] * dz;
        const double dpo0 = s_sum[4] * dz, dpoH = s_sum[5] * dz, dpoa = s_sum[6] * dz, dpob = s_sum[7] * dz;
        double ai1 = kp.rtb * (dpo0 - dpoa) - dpi0;
        double ai2 = kp.rtt * (dpoH - dpob) - dpiH;
        if (kp.sigma_on) {
            ai1 -= kp.sig_hat[0].x / kp.eps;
            ai2 += kp.sig_hat[M].x / kp.eps;
        }
        double Ai;
        if (kp.metal_b && kp.metal_t) Ai = -(piH - pi0) / kp.H;
        else if (kp.metal_b) Ai = ai2;
        else if (kp.metal_t) Ai = ai1;
        else Ai = 0.5 * (ai1 + ai2);
        kp.scal[1] = Ai;
        kp.zcol[2 * N] = s_sum[8];          // gauge term of k = 0: no damping, no correction
        if (kp.sigma_on) {
            kp.scal[7] = s_sum[8];
            kp.scal[8] = s_sum[9] + Ai * kp.H;
        }
    }
}
__global__ void __launch_bounds__(kZeroThreads) k_column_zero(KP kp) { column_zero_body(kp); }

// ---------------------------------------------------------------------------
// The boundary-condition correction of one mode in double (Sec. 4.3.3): from
// the wall values of psi_i*, psi_o* and their z derivatives (16 float sums
// over the coefficients, the last factor 2/Hbar of the derivatives not yet
// applied), the mismatches Eq. (mm1)-(mm4) (with wall charges, the sigma
// terms), the coefficients P, Q of the normalised Eq. (inphisc) and its value
// at z = 0. The factors of k (k, e^{-kH}, 1/den, the z = 0 factor of P) come
// from the plan's extended-precision table kp.mtab.
// ---------------------------------------------------------------------------
struct BcCoef {
    double2 P, Q;
    double corr0;
    double ekH, iden;
};

__device__ __forceinline__ BcCoef bc_correction(const KP& kp, int col, const float* v) {
    const double4_32a t = kp.mtab[col];
    const double dz = 2.0 / kp.Hbar;
    double2 mpb = make_double2(fma(-kp.tb, double(v[8]), double(v[0])), fma(-kp.tb, double(v[9]), double(v[1])));
    double2 meb = make_double2(fma(-kp.rtb, double(v[10]), double(v[2])) * dz,
                               fma(-kp.rtb, double(v[11]), double(v[3])) * dz);
    double2 mpt = make_double2(fma(-kp.tt, double(v[12]), double(v[4])), fma(-kp.tt, double(v[13]), double(v[5])));
    double2 met = make_double2(fma(-kp.rtt, double(v[14]), double(v[6])) * dz,
                               fma(-kp.rtt, double(v[15]), double(v[7])) * dz);
    if (kp.sigma_on) {   // Eq. (mm2), (mm4): +sigma_b, -sigma_t (over eps)
        const double ie = 1.0 / kp.eps;
        meb = cadd(meb, cscale(kp.sig_hat[col], ie));
        met = csub(met, cscale(kp.sig_hat[size_t(kp.ny) * kp.nxh + col], ie));
    }
    const double ik = 1.0 / t.x;
    const double db = kp.db * ik, dt = kp.dt * ik;
    BcCoef o;
    o.P = csub(cscale(mpb, kp.cb), cscale(meb, db));
    o.Q = csub(cscale(mpt, -kp.ct), cscale(met, dt));
    o.ekH = t.y;
    o.iden = t.z;
    o.corr0 = t.w * o.P.x + (t.y * (1.0 - kp.Gb) * t.z) * o.Q.x;
    return o;
}

// wave number of mode col (double) and its weight in the half spectrum
__device__ __forceinline__ double mode_k(const KP& kp, int col, double& mult) {
    const int iy = col / kp.nxh, ix = col - iy * kp.nxh;
    const int my = iy < (kp.ny + 1) / 2 ? iy : iy - kp.ny;
    const double kx = kTwoPi * ix / kp.Lx, ky = kTwoPi * my / kp.Ly;
    mult = (ix == 0 || (kp.nx % 2 == 0 && ix == kp.nx / 2)) ? 1.0 : 2.0;
    return sqrt(kx * kx + ky * ky);
}


// Once per plan: the correction factors of the modes without a correction
// (k = 0 or k > k_max, decided with the wave number in double exactly as the
// FP64 column kernel decides it) are set to zero, keeping k, so that the
// per-solve kernels read the decision from the table (1/den != 0).
__global__ void k_mode_flags(KP kp, double4_32a* mtab) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= kp.ny * kp.nxh) return;
    double mult;
    const double k = mode_k(kp, col, mult);
    if (!(k > 0.0 && k <= kp.kmax)) mtab[col] = make_double4_32a(mtab[col].x, 0.0, 0.0, 0.0);
}

// ---------------------------------------------------------------------------
// Column stage of the tensor-core form (DPSLAB_MIXED with the z transforms as
// GEMMs around it): the per-mode BVP of Appendix A on 8 W modes per block of
// 2 W warps, the boundary-condition correction in double (Sec. 4.3.3)
// inside the block.
//  1. The Chebyshev coefficients of both densities come in as whole rows of
//     the block's modes, scaled to the right-hand side of Eq. (blocksys):
//     F[mode][n] = (f_i, f_o).
//  2. Warp w < W runs the two-way banded sweeps of 8 modes, one lane per
//     (mode, chain, side): A y'' = F and A x = K^2 e0 (e1), A = I - K^2 J^2.
//  3. Every warp then takes modes one at a time, lanes over n = lane + 32 r:
//     the 2 x 2 Schur system for (c, d) of each field, y'' += (c or d) x,
//     then y' = J y'' + d e0 and y = J y' + c e0 for field i (neighbours by
//     shuffles), and the wall values: psi_i*, d psi_i*/dz from y, y'; psi_o*,
//     d psi_o*/dz from y''_o through J^T t and J^T J^T t (t = T_n at the
//     wall), since sum t y = (J^T J^T t).y'' + d (J^T t)_0 + c t_0 and
//     sum t y' = (J^T t).y'' + d t_0.
//  4. One thread per mode: the correction coefficients in double
//     (bc_correction) -> colp, and its gauge term.
//  5. y and y' of field i leave as whole rows, for the node-value GEMM.
// R = ceil(N / 32) values of n per lane (4 for N <= 128, 8 for N <= 256).
// ---------------------------------------------------------------------------
constexpr int kTcTables = 15;   // j2l j2d j2u u1 u2 v1 v2 t0 tH wg hinv jt0 jjt0 jtH jjtH

__host__ __device__ inline int tc_stride(int N) { return N | 1; }   // odd: rows of modes fall in distinct banks

template <int W, int R>
__device__ __forceinline__ void column_tc_body(const KP& kp, const int bid, const bool load_tables = true,
                                               const int next_bid = -1) {
    constexpr int MB = 8 * W;                 // modes per block
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = kp.nz, NP = tc_stride(N);
    const int M = kp.ny * kp.nxh;
    float4* F = reinterpret_cast<float4*>(smraw);                  // [MB][NP]
    float2* Q = reinterpret_cast<float2*>(F + MB * NP);            // [MB][NP]: c' or a'', x
    float* tb = reinterpret_cast<float*>(Q + MB * NP);             // [kTcTables][N]
    const float *j2l = tb, *j2d = tb + N, *j2u = tb + 2 * N, *u1 = tb + 3 * N, *u2 = tb + 4 * N, *v1 = tb + 5 * N,
                *v2 = tb + 6 * N, *t0 = tb + 7 * N, *tH = tb + 8 * N, *wgt = tb + 9 * N, *hinv = tb + 10 * N,
                *jt0 = tb + 11 * N, *jjt0 = tb + 12 * N, *jtH = tb + 13 * N, *jjtH = tb + 14 * N;
    __shared__ float s_K[MB], s_mult[MB], s_damp[MB], s_kf[MB];
    __shared__ float s_bs[MB][16];
    __shared__ double s_gauge[MB];
    __shared__ int s_valid[MB], s_corr[MB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = 2 * W, bs = 32 * NW;   // the first W warps sweep; all take part in the rest
    const int col0 = bid * MB;
    float2* const sp = static_cast<float2*>(kp.spec);

    if (tid < MB) {
        // wave number from the plan's factor table (whose zero factors mark
        // the modes without a correction: k = 0 or k > k_max)
        const int c = tid, col = col0 + c;
        const int iy = col / kp.nxh, ix = col - iy * kp.nxh;
        const double4_32a t = col < M ? kp.mtab[col] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
        const float k = float(t.x);
        s_valid[c] = col < M;
        s_kf[c] = k;
        s_K[c] = float(0.5 * t.x * kp.Hbar);
        s_mult[c] = (ix == 0 || (kp.nx % 2 == 0 && ix == kp.nx / 2)) ? 1.f : 2.f;
        s_damp[c] = expf(-0.5f * kp.f.sigma2 * k * k);
        s_corr[c] = t.z != 0.0;
        s_gauge[c] = 0.0;
    }
    if (load_tables) {
        // the tables into shared memory (once per block: a persistent block
        // keeps them for all its blocks of modes); every load of a batch of 8
        // is issued before the first store (one round trip per batch)
        const float* src[kTcTables] = {kp.j2l32, kp.j2d32, kp.j2u32, kp.u132, kp.u232, kp.v132, kp.v232, kp.t032,
                                       kp.tH32, kp.wg32, kp.hinv32, kp.jt0_32, kp.jjt0_32, kp.jtH_32, kp.jjtH_32};
        for (int t0b = tid; t0b < kTcTables * N; t0b += 8 * bs) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t0b + u * bs;
                v[u] = t < kTcTables * N ? __ldg(src[t / N] + t % N) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t0b + u * bs;
                if (t < kTcTables * N) tb[t] = v[u];
            }
        }
    }
    // 1. coefficients of both densities, whole rows of the block's modes;
    //    every load of a batch is issued before the first store
    const float scale = kp.f.scale;
    constexpr int kLd = 4;
    for (int t0 = tid; t0 < N * MB; t0 += kLd * bs) {
        float2 vi[kLd], vo[kLd];
#pragma unroll
        for (int u = 0; u < kLd; ++u) {
            const int t = t0 + u * bs, n = t / MB, c = t - n * MB, col = col0 + c;
            vi[u] = vo[u] = make_float2(0.f, 0.f);
            if (t < N * MB && col < M) {
                vi[u] = __ldcs(sp + size_t(n) * M + col);
                vo[u] = __ldcs(sp + size_t(N + n) * M + col);
            }
        }
#pragma unroll
        for (int u = 0; u < kLd; ++u) {
            const int t = t0 + u * bs, n = t / MB, c = t - n * MB;
            if (t < N * MB) F[c * NP + n] = make_float4(vi[u].x * scale, vi[u].y * scale, vo[u].x * scale, vo[u].y * scale);
        }
    }
    // the next block of modes of a persistent block: its coefficient rows
    // (both spectra, 128-byte lines) into L2 while this block computes
    if (next_bid >= 0) {
        constexpr int kLines = (MB * 8 + 127) / 128;
        const int ncol0 = next_bid * MB;
        for (int i = tid; i < 2 * N * kLines; i += bs) {
            const int row = i / kLines, c = ncol0 + (i - row * kLines) * 16;
            if (c < M) asm volatile("prefetch.global.L2 [%0];" ::"l"(sp + size_t(row) * M + c));
        }
    }
    // 1b. rho_o's coefficients from its node values at the pairs (a, m - a)
    //     it can reach (Sec. 5.2.2 step 3, the DCT-I form): S = v_a + v_{m-a}
    //     and D = v_a - v_{m-a} per mode and pair (staged where the sweeps'
    //     Q goes), then coefficient n = sum_p o_fwd[p][n] (S_p or D_p by the
    //     parity of n), threads over consecutive n
    __syncthreads();

    // 2. two-way banded sweeps: lane (mode c, chain ch, side) of warp w < W. Side
    //    0 sweeps rows 0 .. m-1 downward (row i becomes y_i + c'_i y_{i+1} =
    //    f'_i), side 1 rows L-1 .. m upward (a''_i y_{i-1} + y_i = f''_i);
    //    they meet in a 2 x 2 system at rows m-1, m, then substitute outward.
    if (warp < W) {
        const int c = 8 * warp + (lane >> 2), ch = (lane >> 1) & 1, side = lane & 1;
        const float K2 = s_K[c] * s_K[c];
        float4* Fc = F + c * NP;
        float2* Qc = Q + c * NP;
        const int L = (N - ch + 1) / 2, m = L / 2;
        const int cnt = side ? L - m : m, i0 = side ? L - 1 : 0, di = side ? -1 : 1;
        const int cmax = L - m;
        float qp = 0.f, xcp = 0.f;
        float4 fp = make_float4(0.f, 0.f, 0.f, 0.f);
        int nn = ch + 2 * i0;
        float jl = 0.f, jd = 0.f, ju = 0.f;
        float4 Fn = fp;
        if (cnt > 0) { jl = j2l[nn]; jd = j2d[nn]; ju = j2u[nn]; Fn = Fc[nn]; }
        for (int k = 0; k < cmax; ++k) {
            if (k < cnt) {
                const int i = i0 + di * k, n = nn;
                const float an = -K2 * jl, bn = 1.f - K2 * jd, cn = -K2 * ju;
                const float4 Fcur = Fn;
                nn = n + 2 * di;
                if (k + 1 < cnt) { jl = j2l[nn]; jd = j2d[nn]; ju = j2u[nn]; Fn = Fc[nn]; }
                const float lo = side ? cn : an, up = side ? an : cn;   // toward / away from the sweep
                const float inv = __frcp_rn(bn - lo * qp);
                const float rn = (i == 0) ? K2 : 0.f;
                fp = make_float4((Fcur.x - fp.x * lo) * inv, (Fcur.y - fp.y * lo) * inv, (Fcur.z - fp.z * lo) * inv,
                                 (Fcur.w - fp.w * lo) * inv);
                xcp = (rn - lo * xcp) * inv;
                qp = up * inv;
                Qc[n] = make_float2(qp, xcp);
                Fc[n] = fp;
            }
        }
        __syncwarp();
        if (side == 1 && m > 0) {
            const int nA = ch + 2 * (m - 1), nB = ch + 2 * m;
            const float2 qA = Qc[nA], qB = Qc[nB];
            const float cA = qA.x, aB = qB.x;
            const float den = 1.f / (1.f - aB * cA);
            const float4 FA = Fc[nA], FB = Fc[nB];
            const float4 yB = make_float4((FB.x - aB * FA.x) * den, (FB.y - aB * FA.y) * den, (FB.z - aB * FA.z) * den,
                                          (FB.w - aB * FA.w) * den);
            const float yBx = (qB.y - aB * qA.y) * den;
            Fc[nA] = make_float4(FA.x - cA * yB.x, FA.y - cA * yB.y, FA.z - cA * yB.z, FA.w - cA * yB.w);
            Qc[nA] = make_float2(cA, qA.y - cA * yBx);
            Fc[nB] = yB;
            Qc[nB] = make_float2(aB, yBx);
        }
        __syncwarp();
        const int bcnt = side ? L - m - 1 : m - 1, b0 = side ? m + 1 : m - 2, bdi = -di;
        if (bcnt > 0) {
            const int nprev = ch + 2 * (b0 - bdi);
            fp = Fc[nprev];
            xcp = Qc[nprev].y;
        }
        for (int k = 0; k < cmax; ++k) {
            if (k < bcnt) {
                const int i = b0 + bdi * k, n = ch + 2 * i;
                const float2 qn = Qc[n];
                const float4 Fv = Fc[n];
                fp = make_float4(Fv.x - qn.x * fp.x, Fv.y - qn.x * fp.y, Fv.z - qn.x * fp.z, Fv.w - qn.x * fp.w);
                xcp = qn.y - qn.x * xcp;
                Fc[n] = fp;
                Qc[n] = make_float2(qn.x, xcp);
            }
        }
    }
    __syncthreads();

    // 3. per mode, lanes over n = lane + 32 r
    for (int c = warp; c < MB; c += NW) {
        const float K = s_K[c];
        float2 yi[R], yo[R];
        float x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int n = lane + 32 * r;
            yi[r] = yo[r] = make_float2(0.f, 0.f);
            x[r] = 0.f;
            if (n < N) {
                const float4 f = F[c * NP + n];
                yi[r] = make_float2(f.x, f.y);
                yo[r] = make_float2(f.z, f.w);
                x[r] = Q[c * NP + n].y;
            }
        }
        // Schur rows (Eq. (BCs); Eq. (BCs0) for K = 0): sums of g_t, g_b times
        // y'' of both fields and times x (by the parity of n = that of lane)
        float da[12];
        {
            float acc[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) acc[i] = 0.f;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int n = lane + 32 * r;
                if (n < N) {
                    const float gtn = K > 0.f ? u1[n] + K * u2[n] : u2[n];
                    const float gbn = K > 0.f ? v1[n] - K * v2[n] : v2[n];
                    acc[0] = fmaf(gtn, yi[r].x, acc[0]); acc[1] = fmaf(gtn, yi[r].y, acc[1]);
                    acc[2] = fmaf(gbn, yi[r].x, acc[2]); acc[3] = fmaf(gbn, yi[r].y, acc[3]);
                    acc[4] = fmaf(gtn, yo[r].x, acc[4]); acc[5] = fmaf(gtn, yo[r].y, acc[5]);
                    acc[6] = fmaf(gbn, yo[r].x, acc[6]); acc[7] = fmaf(gbn, yo[r].y, acc[7]);
                    if (lane & 1) { acc[9] = fmaf(gtn, x[r], acc[9]); acc[11] = fmaf(gbn, x[r], acc[11]); }
                    else { acc[8] = fmaf(gtn, x[r], acc[8]); acc[10] = fmaf(gbn, x[r], acc[10]); }
                }
            }
            const float r8 = warp_sum_multi<8>(acc), r4 = warp_sum_multi<4>(acc + 8);
#pragma unroll
            for (int i = 0; i < 8; ++i) da[i] = __shfl_sync(0xffffffffu, r8, 4 * i);
#pragma unroll
            for (int i = 0; i < 4; ++i) da[8 + i] = __shfl_sync(0xffffffffu, r4, 8 * i);
        }
        float2 cc[2], dd[2];
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const float2 sFt = f ? make_float2(da[4], da[5]) : make_float2(da[0], da[1]);
            const float2 sFb = f ? make_float2(da[6], da[7]) : make_float2(da[2], da[3]);
            if (K > 0.f) {
                const float m11 = K + da[8], m12 = 1.f + K + da[9], m21 = -K + da[10], m22 = 1.f + K + da[11];
                const float idet = 1.f / (m11 * m22 - m12 * m21);
                cc[f] = cscale(csub(cscale(sFt, m22), cscale(sFb, m12)), -idet);
                dd[f] = cscale(csub(cscale(sFb, m11), cscale(sFt, m21)), -idet);
            } else {
                cc[f] = cscale(cadd(sFt, sFb), -0.5f);
                dd[f] = cscale(csub(sFt, sFb), -0.5f);
            }
        }
        // y'' = x_F + c x_c + d x_d (c on even n, d on odd n)
        {
            const float2 mi = (lane & 1) ? dd[0] : cc[0], mo = (lane & 1) ? dd[1] : cc[1];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                yi[r] = cadd(yi[r], cscale(mi, x[r]));
                yo[r] = cadd(yo[r], cscale(mo, x[r]));
            }
        }
        // y' = J y'' + d e0 and y = J y' + c e0 for field i: entry n of J v is
        // (v_{n-1} - v_{n+1}) / (2n) for n >= 2 and v_0 - v_2 / 2 for n = 1;
        // v_{n-1} and v_{n+1} from the neighbouring lanes (lane 0 takes lane
        // 31's value of row r - 1, lane 31 lane 0's of row r + 1)
        auto integrate = [&](const float2* v, float2* out, float2 e0) {
            // rotations by one lane: lane 0 takes lane 31's value of the row
            // before (the previous row's rotation), lane 31 lane 0's of the
            // row after (the next row's)
            float2 pr[R], nr[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                pr[r].x = __shfl_sync(0xffffffffu, v[r].x, (lane + 31) & 31);
                pr[r].y = __shfl_sync(0xffffffffu, v[r].y, (lane + 31) & 31);
                nr[r].x = __shfl_sync(0xffffffffu, v[r].x, (lane + 1) & 31);
                nr[r].y = __shfl_sync(0xffffffffu, v[r].y, (lane + 1) & 31);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int n = lane + 32 * r;
                const float2 prev = lane != 0 ? pr[r] : (r > 0 ? pr[r - 1] : make_float2(0.f, 0.f));
                float2 next = lane != 31 ? nr[r] : (r + 1 < R ? nr[r + 1] : make_float2(0.f, 0.f));
                if (n + 1 >= N) next = make_float2(0.f, 0.f);
                float2 o;
                if (n == 0) o = e0;
                else if (n == 1) o = csub(prev, cscale(next, 0.5f));
                else o = cscale(csub(prev, next), hinv[n < N ? n : 0]);
                out[r] = n < N ? o : make_float2(0.f, 0.f);
            }
        };
        float2 ypi[R], yyi[R];
        integrate(yi, ypi, dd[0]);
        integrate(ypi, yyi, cc[0]);
        // wall values: values 0..15 in the order of bc_correction, 16-17 the
        // gauge sum of psi_i*
        float acc[18];
#pragma unroll
        for (int i = 0; i < 18; ++i) acc[i] = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int n = lane + 32 * r;
            if (n < N) {
                const float a0 = t0[n], aH = tH[n];
                acc[0] = fmaf(a0, yyi[r].x, acc[0]);   acc[1] = fmaf(a0, yyi[r].y, acc[1]);
                acc[2] = fmaf(a0, ypi[r].x, acc[2]);   acc[3] = fmaf(a0, ypi[r].y, acc[3]);
                acc[4] = fmaf(aH, yyi[r].x, acc[4]);   acc[5] = fmaf(aH, yyi[r].y, acc[5]);
                acc[6] = fmaf(aH, ypi[r].x, acc[6]);   acc[7] = fmaf(aH, ypi[r].y, acc[7]);
                acc[8] = fmaf(jjt0[n], yo[r].x, acc[8]);  acc[9] = fmaf(jjt0[n], yo[r].y, acc[9]);
                acc[10] = fmaf(jt0[n], yo[r].x, acc[10]); acc[11] = fmaf(jt0[n], yo[r].y, acc[11]);
                acc[12] = fmaf(jjtH[n], yo[r].x, acc[12]); acc[13] = fmaf(jjtH[n], yo[r].y, acc[13]);
                acc[14] = fmaf(jtH[n], yo[r].x, acc[14]); acc[15] = fmaf(jtH[n], yo[r].y, acc[15]);
                acc[16] = fmaf(wgt[n], yyi[r].x, acc[16]); acc[17] = fmaf(wgt[n], yyi[r].y, acc[17]);
            }
        }
        // lane 2 v holds value v (0..15); lane 16 v holds value 16 + v
        float r16 = warp_sum_multi<16>(acc);
        const float r2 = warp_sum_multi<2>(acc + 16);
        {
            // the (c, d) terms of field o's wall values
            const int v = lane >> 1, comp = v & 1;
            const float co = comp ? cc[1].y : cc[1].x, dv = comp ? dd[1].y : dd[1].x;
            if (v == 8 || v == 9) r16 += dv * jt0[0] + co * t0[0];
            else if (v == 10 || v == 11) r16 += dv * t0[0];
            else if (v == 12 || v == 13) r16 += dv * jtH[0] + co * tH[0];
            else if (v == 14 || v == 15) r16 += dv * tH[0];
        }
        const float wgs = __shfl_sync(0xffffffffu, r2, 0);
        if (s_corr[c] && (lane & 1) == 0) s_bs[c][lane >> 1] = r16;
        if (lane == 0 && s_valid[c]) s_gauge[c] = double(s_mult[c]) * double(s_damp[c]) * double(wgs);
        // y and y' of field i, for the node-value GEMM
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int n = lane + 32 * r;
            if (n < N) F[c * NP + n] = make_float4(yyi[r].x, yyi[r].y, ypi[r].x, ypi[r].y);
        }
    }
    __syncthreads();

    // column 0 (block 0): the coefficients and gauge term of k_column_zero
    if (bid == 0) {
        for (int n = tid; n < N; n += bs) F[n] = make_float4(float(kp.zcol[n]), 0.f, float(kp.zcol[N + n]), 0.f);
        if (tid == 0) s_gauge[0] = kp.zcol[2 * N];
        __syncthreads();
    }
    // 4. the correction coefficients in double, one thread per mode (while
    //    the other warps store)
    if (tid < MB) {
        const int c = tid, col = col0 + c;
        if (s_valid[c]) {
            const float k = s_kf[c];
            const double mult = s_mult[c];
            ColP cp{make_float2(0.f, 0.f), make_float2(0.f, 0.f), k, 0.f, 0.f, 0};
            if (s_corr[c]) {
                const BcCoef b = bc_correction(kp, col, s_bs[c]);
                cp = ColP{make_float2(float(b.P.x), float(b.P.y)), make_float2(float(b.Q.x), float(b.Q.y)), k,
                          float(b.ekH), float(b.iden), 1};
                s_gauge[c] += mult * b.corr0;
            }
            kp.colp[col] = cp;
        }
    }
    // 5. coefficients of psi_i (plane 0) and dpsi_i/dz (plane 1, before the
    //    factor 2/Hbar), whole rows
    for (int t = tid; t < 2 * N * MB; t += bs) {
        const int c = t % MB, fn = t / MB, col = col0 + c;
        const int f = fn >= N, n = fn - f * N;
        if (col < M) {
            const float4 v = F[c * NP + n];
            __stcs(sp + size_t(fn) * M + col, f ? make_float2(v.z, v.w) : make_float2(v.x, v.y));
        }
    }
    __syncthreads();
    if (tid == 0) {
        double g = 0.0;
        for (int c = 0; c < MB; ++c) g += s_gauge[c];
        kp.part_gauge_far[bid] = g;
    }
}

template <int W, int R>
// persistent: as many blocks as fit on the device, each taking blocks of
// modes bid, bid + gridDim.x, ... and loading the tables once
__global__ void __launch_bounds__(64 * W, 2) k_column_tc(KP kp) {
    for (int bid = blockIdx.x; bid < kp.n_col_blocks; bid += gridDim.x) {
        const int next = bid + int(gridDim.x);
        column_tc_body<W, R>(kp, bid, bid == int(blockIdx.x), next < kp.n_col_blocks ? next : -1);
        __syncthreads();
    }
}
template <int W, int R>
__global__ void __launch_bounds__(64 * W, 2) k_column_tc_batch(const __grid_constant__ ColBatch b) {
    const int s = batch_system(b.starts, b.nsys, blockIdx.x);
    column_tc_body<W, R>(b.kp[s], blockIdx.x - b.starts[s]);
}

// ---------------------------------------------------------------------------
// Mixed-precision column kernel (DPSLAB_MIXED): the same steps as k_column
// with the transforms, the banded solve, the Schur 2x2 systems, the boundary
// values and the node values in float; the mismatches, the correction
// coefficients and the gauge sum in double; the k = 0 column (coefficients,
// slope, gauge term) taken from k_column_zero, which solves it in double.
// The correction is evaluated at the nodes in float: its normalised form
// only multiplies decaying factors bounded by e^{k_max H_E}, far inside
// float range.
// ---------------------------------------------------------------------------
constexpr int kColBlockM = 8;
constexpr int kColThreadsM = 32 * kColBlockM;

// kTensor: the z transforms run as tensor-core GEMMs around this kernel
// (k_zgemm); it then reads the coefficients of both densities and writes
// the coefficients of psi_i and dpsi_i/dz and each mode's correction
// parameters, instead of transforming itself.
template <int CB>
__device__ __forceinline__ void column_mixed_body(const KP& kp, const int bid) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = kp.nz;
    // padded column stride, NP = 2 mod 16: eight modes x two rows of float2
    // (the mode-major loads and stores) then fall in distinct banks
    const int NP = N + ((2 - N) & 15);
    const int M = kp.ny * kp.nxh;
    float2* Vi = reinterpret_cast<float2*>(smraw);
    float2* Vo = Vi + CB * NP;
    float2* Ci = Vo + CB * NP;
    float2* Co = Ci + CB * NP;
    float* cpv = reinterpret_cast<float*>(Co + CB * NP);
    float* xe = cpv + CB * NP;
    __shared__ float s_k[CB], s_K[CB], s_mult[CB], s_iden[CB], s_ekH[CB];
    __shared__ float s_bs[CB][16];
    __shared__ double s_gauge[CB];
    __shared__ int s_valid[CB], s_corr[CB];
    __shared__ float2 s_c[2][CB], s_d[2][CB], s_P[CB], s_Q[CB];
    __shared__ double s_Ai;
    const int tid = threadIdx.x, bs = blockDim.x;
    const int col0 = bid * CB;
    float2* const sp = static_cast<float2*>(kp.spec);

    if (tid < CB) {
        const int c = tid, col = col0 + c;
        const int iy = col / kp.nxh, ix = col - iy * kp.nxh;
        const int my = iy < (kp.ny + 1) / 2 ? iy : iy - kp.ny;
        const double kx = kTwoPi * ix / kp.Lx, ky = kTwoPi * my / kp.Ly;
        const double k = sqrt(kx * kx + ky * ky);
        s_valid[c] = col < M;
        s_k[c] = float(k);
        s_K[c] = float(0.5 * k * kp.Hbar);
        s_mult[c] = (ix == 0 || (kp.nx % 2 == 0 && ix == kp.nx / 2)) ? 1.f : 2.f;
        s_corr[c] = (col < M) && k > 0.0 && k <= kp.kmax;
        s_gauge[c] = 0.0;
    }
    // the k = 0 slope, from k_column_zero (block 0 holds column 0)
    if (tid == 0) s_Ai = bid == 0 ? kp.scal[1] : 0.0;
    const float scale = kp.f.scale;
    // every load of a batch is issued before the first store: one memory
    // round trip per batch instead of one per row group
    constexpr int kLd = 4;
    for (int t0 = tid; t0 < N * CB; t0 += kLd * bs) {
        float2 vi[kLd], vo[kLd];
#pragma unroll
        for (int u = 0; u < kLd; ++u) {
            const int t = t0 + u * bs, j = t / CB, c = t - j * CB, col = col0 + c;
            vi[u] = vo[u] = make_float2(0.f, 0.f);
            if (t < N * CB && col < M) {
                vi[u] = __ldcs(sp + size_t(j) * M + col);
                vo[u] = __ldcs(sp + size_t(N + j) * M + col);
            }
        }
#pragma unroll
        for (int u = 0; u < kLd; ++u) {
            const int t = t0 + u * bs, j = t / CB, c = t - j * CB;
            if (t >= N * CB) break;
            Vi[c * NP + j] = vi[u];
            Vo[c * NP + j] = vo[u];
        }
    }
    __syncthreads();

    const int m = N - 1, JE = (N + 1) / 2, JO = N / 2;
    {
    for (int t = tid; t < 2 * CB * JE; t += bs) {
        const int f = t / (CB * JE), r = t - f * CB * JE, c = r / JE, a = r - c * JE;
        if (a < m - a) {
            float2* V = (f ? Vo : Vi) + c * NP;
            const float2 va = V[a], vb = V[m - a];
            V[a] = cadd(va, vb);
            V[m - a] = csub(va, vb);
        }
    }
    __syncthreads();
    // one thread per output row q for all CB modes: each table entry feeds
    // 4 CB multiply-adds (the node values are shared-memory broadcasts)
    for (int q = tid; q < N; q += bs) {
        const bool odd = q >= JE;
        const int na = odd ? JO : JE;
        float acc[CB][4];
#pragma unroll
        for (int c = 0; c < CB; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.f;
        for (int a = 0; a < na; ++a) {
            const float w = kp.cft32[size_t(a) * N + q];
            const int ia = odd ? m - a : a;
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const float2 u = Vi[c * NP + ia], v = Vo[c * NP + ia];
                acc[c][0] = fmaf(w, u.x, acc[c][0]);
                acc[c][1] = fmaf(w, u.y, acc[c][1]);
                acc[c][2] = fmaf(w, v.x, acc[c][2]);
                acc[c][3] = fmaf(w, v.y, acc[c][3]);
            }
        }
        const int n = odd ? 2 * (q - JE) + 1 : 2 * q;
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            Ci[c * NP + n] = make_float2(acc[c][0] * scale, acc[c][1] * scale);
            Co[c * NP + n] = make_float2(acc[c][2] * scale, acc[c][3] * scale);
        }
    }
    __syncthreads();
    }

    // Appendix A banded solve (even and odd chains), float, eliminated from
    // both ends at once: lane side 0 sweeps rows 0 .. m-1 downward (row i
    // becomes y_i + c'_i y_{i+1} = f'_i), lane side 1 sweeps rows L-1 .. m
    // upward (a''_i y_{i-1} + y_i = f''_i); the two meet in a 2 x 2 system at
    // rows m-1, m, then substitute back outward. One instruction stream for
    // both directions (per-lane start, step and coefficient roles). The
    // 4 CB lanes of warp 0: (mode c, chain ch, side).
    static_assert(4 * CB <= 32, "the two-way sweeps run in one warp");
    // the lanes of warp 0 that take part (all of it for 8 modes per block)
    constexpr unsigned kSweepLanes = 4 * CB == 32 ? 0xffffffffu : (1u << (4 * CB)) - 1u;
    if (tid < 4 * CB) {
        const int c = tid >> 2, ch = (tid >> 1) & 1, side = tid & 1;
        const float K2 = s_K[c] * s_K[c];
        float2* Fi = Ci + c * NP;
        float2* Fo = Co + c * NP;
        float* cq = cpv + c * NP;          // c'_i (side 0 rows), a''_i (side 1 rows)
        float* xc = xe + c * NP;
        const int L = (N - ch + 1) / 2, m = L / 2;
        const int cnt = side ? L - m : m, i0 = side ? L - 1 : 0, di = side ? -1 : 1;
        const int cmax = L - m;            // >= m: the longer sweep
        float qp = 0.f, xcp = 0.f;
        float2 fip = make_float2(0.f, 0.f), fop = fip;
        int nn = ch + 2 * i0;
        float jl = 0.f, jd = 0.f, ju = 0.f;
        float2 Fin = make_float2(0.f, 0.f), Fon = Fin;
        if (cnt > 0) { jl = kp.j2l32[nn]; jd = kp.j2d32[nn]; ju = kp.j2u32[nn]; Fin = Fi[nn]; Fon = Fo[nn]; }
        for (int k = 0; k < cmax; ++k) {
            if (k < cnt) {
                const int i = i0 + di * k, n = nn;
                // the band tables are zero below row 2 and above row N - 3
                const float an = -K2 * jl;
                const float bn = 1.f - K2 * jd;
                const float cn = -K2 * ju;
                const float2 Fcur = Fin, Focur = Fon;
                nn = n + 2 * di;
                if (k + 1 < cnt) { jl = kp.j2l32[nn]; jd = kp.j2d32[nn]; ju = kp.j2u32[nn]; Fin = Fi[nn]; Fon = Fo[nn]; }
                const float lo = side ? cn : an, up = side ? an : cn;   // toward / away from the sweep
                const float inv = __frcp_rn(bn - lo * qp);
                const float rn = (i == 0) ? K2 : 0.f;
                fip = cscale(csub(Fcur, cscale(fip, lo)), inv);
                fop = cscale(csub(Focur, cscale(fop, lo)), inv);
                xcp = (rn - lo * xcp) * inv;
                qp = up * inv;
                cq[n] = qp;
                Fi[n] = fip;
                Fo[n] = fop;
                xc[n] = xcp;
            }
        }
        __syncwarp(kSweepLanes);
        if (side == 1 && m > 0) {
            // rows m-1 (y + c' y_m = f') and m (a'' y_{m-1} + y = f'')
            const int nA = ch + 2 * (m - 1), nB = ch + 2 * m;
            const float cA = cq[nA], aB = cq[nB];
            const float den = 1.f / (1.f - aB * cA);
            const float2 yBi = cscale(csub(Fi[nB], cscale(Fi[nA], aB)), den);
            const float2 yBo = cscale(csub(Fo[nB], cscale(Fo[nA], aB)), den);
            const float yBx = (xc[nB] - aB * xc[nA]) * den;
            Fi[nA] = csub(Fi[nA], cscale(yBi, cA));
            Fo[nA] = csub(Fo[nA], cscale(yBo, cA));
            xc[nA] = xc[nA] - cA * yBx;
            Fi[nB] = yBi;
            Fo[nB] = yBo;
            xc[nB] = yBx;
        }
        __syncwarp(kSweepLanes);
        // substitute outward from the interface: side 0 rows m-2 .. 0,
        // side 1 rows m+1 .. L-1
        const int bcnt = side ? L - m - 1 : m - 1, b0 = side ? m + 1 : m - 2, bdi = -di;
        if (bcnt > 0) {
            const int nprev = ch + 2 * (b0 - bdi);
            fip = Fi[nprev];
            fop = Fo[nprev];
            xcp = xc[nprev];
        }
        for (int k = 0; k < cmax; ++k) {
            if (k < bcnt) {
                const int i = b0 + bdi * k, n = ch + 2 * i;
                const float q = cq[n];
                fip = csub(Fi[n], cscale(fip, q));
                fop = csub(Fo[n], cscale(fop, q));
                xcp = xc[n] - q * xcp;
                Fi[n] = fip;
                Fo[n] = fop;
                xc[n] = xcp;
            }
        }
    }
    __syncthreads();

    // Schur 2x2 (warp per column, float)
    {
        const int c = tid >> 5, lane = tid & 31;
        const float K = s_K[c];
        const float2* Xi = Ci + c * NP;
        const float2* Xo = Co + c * NP;
        const float* xc = xe + c * NP;
        float acc[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int n = lane; n < N; n += 32) {
            const float gtn = K > 0.f ? kp.u132[n] + K * kp.u232[n] : kp.u232[n];
            const float gbn = K > 0.f ? kp.v132[n] - K * kp.v232[n] : kp.v232[n];
            acc[0] = fmaf(gtn, Xi[n].x, acc[0]); acc[1] = fmaf(gtn, Xi[n].y, acc[1]);
            acc[2] = fmaf(gbn, Xi[n].x, acc[2]); acc[3] = fmaf(gbn, Xi[n].y, acc[3]);
            acc[4] = fmaf(gtn, Xo[n].x, acc[4]); acc[5] = fmaf(gtn, Xo[n].y, acc[5]);
            acc[6] = fmaf(gbn, Xo[n].x, acc[6]); acc[7] = fmaf(gbn, Xo[n].y, acc[7]);
            if (n & 1) { acc[9] = fmaf(gtn, xc[n], acc[9]); acc[11] = fmaf(gbn, xc[n], acc[11]); }
            else { acc[8] = fmaf(gtn, xc[n], acc[8]); acc[10] = fmaf(gbn, xc[n], acc[10]); }
        }
        // the 12 sums: values 0..7 (lane 4 v holds value v) and 8..11
        // (lane 8 v holds value 8 + v), gathered where they are used
        const float r8 = warp_sum_multi<8>(acc), r4 = warp_sum_multi<4>(acc + 8);
        float da[12];
#pragma unroll
        for (int i = 0; i < 8; ++i) da[i] = __shfl_sync(0xffffffffu, r8, 4 * i);
#pragma unroll
        for (int i = 0; i < 4; ++i) da[8 + i] = __shfl_sync(0xffffffffu, r4, 8 * i);
        if (lane < 2) {
            const int f = lane;
            const float2 sFt = f ? make_float2(da[4], da[5]) : make_float2(da[0], da[1]);
            const float2 sFb = f ? make_float2(da[6], da[7]) : make_float2(da[2], da[3]);
            float2 cc, dd;
            if (K > 0.f) {
                const float m11 = K + da[8], m12 = 1.f + K + da[9], m21 = -K + da[10], m22 = 1.f + K + da[11];
                const float idet = 1.f / (m11 * m22 - m12 * m21);
                cc = cscale(csub(cscale(sFt, m22), cscale(sFb, m12)), -idet);
                dd = cscale(csub(cscale(sFb, m11), cscale(sFt, m21)), -idet);
            } else {
                cc = cscale(cadd(sFt, sFb), -0.5f);
                dd = cscale(csub(sFt, sFb), -0.5f);
            }
            s_c[f][c] = cc;
            s_d[f][c] = dd;
        }
    }
    // from here to the boundary values warp w works on mode w alone, so
    // warp barriers suffice
    // (blocks of 32 CB threads: one warp per mode of the block)
    __syncwarp();
    // both fields of the warp's mode, n over the lanes: X += (c or d) xe
    // gives y'', then y' = J y'' + d e0 and y = J y' + c e0 (Appendix A
    // integration: entry n of J v is (v_{n-1} - v_{n+1})/(2n), entry 1 is
    // v_0 - v_2/2)
    {
        const int lane_id = tid & 31, c = tid >> 5;
        for (int f = 0; f < 2; ++f) {
            float2* X = (f ? Co : Ci) + c * NP;
            float2* V = (f ? Vo : Vi) + c * NP;
            const float2 mc = s_c[f][c], md = s_d[f][c];
            for (int n = lane_id; n < N; n += 32) X[n] = cadd(X[n], cscale((n & 1) ? md : mc, xe[c * NP + n]));
            __syncwarp();
            for (int n = lane_id; n < N; n += 32) {
                float2 v;
                if (n == 0) v = md;
                else if (n == 1) v = csub(X[0], cscale(X[2], 0.5f));
                else v = cscale(csub(X[n - 1], n + 1 < N ? X[n + 1] : make_float2(0.f, 0.f)), kp.hinv32[n]);
                V[n] = v;
            }
            __syncwarp();
            for (int n = lane_id; n < N; n += 32) {
                float2 v;
                if (n == 0) v = mc;
                else if (n == 1) v = csub(V[0], cscale(V[2], 0.5f));
                else v = cscale(csub(V[n - 1], n + 1 < N ? V[n + 1] : make_float2(0.f, 0.f)), kp.hinv32[n]);
                X[n] = v;
            }
            __syncwarp();
        }
    }

    // boundary values of psi_i*, psi_o* and their z derivatives at the walls
    // (float sums over the coefficients); from them, in double
    // (bc_correction), the mismatches Eq. (mm1)-(mm4) and the correction
    // coefficients of Eq. (inphisc): here for the CUDA-core form, in
    // k_bc_correction for the tensor-core form. The k = 0 column comes from
    // k_column_zero.
    {
        const int c = tid >> 5, lane = tid & 31;
        const float2 *yi = Ci + c * NP, *ypi = Vi + c * NP, *yo = Co + c * NP, *ypo = Vo + c * NP;
        float acc[18];
        for (int i = 0; i < 18; ++i) acc[i] = 0.f;
        for (int n = lane; n < N; n += 32) {
            const float a0 = kp.t032[n], aH = kp.tH32[n], wg = kp.wg32[n];
            acc[0] = fmaf(a0, yi[n].x, acc[0]);   acc[1] = fmaf(a0, yi[n].y, acc[1]);
            acc[2] = fmaf(a0, ypi[n].x, acc[2]);  acc[3] = fmaf(a0, ypi[n].y, acc[3]);
            acc[4] = fmaf(aH, yi[n].x, acc[4]);   acc[5] = fmaf(aH, yi[n].y, acc[5]);
            acc[6] = fmaf(aH, ypi[n].x, acc[6]);  acc[7] = fmaf(aH, ypi[n].y, acc[7]);
            acc[8] = fmaf(a0, yo[n].x, acc[8]);   acc[9] = fmaf(a0, yo[n].y, acc[9]);
            acc[10] = fmaf(a0, ypo[n].x, acc[10]); acc[11] = fmaf(a0, ypo[n].y, acc[11]);
            acc[12] = fmaf(aH, yo[n].x, acc[12]); acc[13] = fmaf(aH, yo[n].y, acc[13]);
            acc[14] = fmaf(aH, ypo[n].x, acc[14]); acc[15] = fmaf(aH, ypo[n].y, acc[15]);
            acc[16] = fmaf(wg, yi[n].x, acc[16]); acc[17] = fmaf(wg, yi[n].y, acc[17]);
        }
        // the 18 sums: values 0..15 (lane 2 v holds value v) and 16, 17
        // (lane 16 v holds value 16 + v)
        const float r16 = warp_sum_multi<16>(acc), r2 = warp_sum_multi<2>(acc + 16);
        const float wgs = __shfl_sync(0xffffffffu, r2, 0);
        if (s_valid[c] && s_corr[c] && (lane & 1) == 0) {
            s_bs[c][lane >> 1] = r16;
        }
        if (lane == 0 && s_valid[c]) {
            const double damp = double(expf(-0.5f * kp.f.sigma2 * s_k[c] * s_k[c]));
            s_gauge[c] = (col0 + c == 0) ? kp.zcol[2 * N] : double(s_mult[c]) * damp * double(wgs);
        }
    }
    {
        // the correction of the block's modes in double, one lane each
        __syncthreads();
        if (tid < CB && s_valid[tid] && s_corr[tid]) {
            const int c = tid;
            const BcCoef b = bc_correction(kp, col0 + c, s_bs[c]);
            s_P[c] = make_float2(float(b.P.x), float(b.P.y));
            s_Q[c] = make_float2(float(b.Q.x), float(b.Q.y));
            s_ekH[c] = float(b.ekH);
            s_iden[c] = float(b.iden);
            s_gauge[c] += double(s_mult[c]) * b.corr0;
        }
    }
    __syncthreads();
    if (bid == 0) {
        // column 0: the coefficients of psi_i and dpsi_i/dz solved in double
        for (int n = tid; n < N; n += bs) {
            Ci[n] = make_float2(float(kp.zcol[n]), 0.f);
            Vi[n] = make_float2(float(kp.zcol[N + n]), 0.f);
        }
        __syncthreads();
    }

    // node values (float), correction at the nodes (float)
    const float Ai = float(s_Ai);
    const float Gb = kp.f.Gb, Gt = kp.f.Gt, Hf = kp.f.H, HEf = kp.f.HE;
    // one thread per node pair a for half the modes at a time: each table
    // entry feeds 4 (CB/2) multiply-adds
    constexpr int CH = CB / 2;
    for (int t = tid; t < 2 * JE; t += bs) {
        const int half = t / JE, a = t - half * JE;
        float ev[CH][4], od[CH][4];
#pragma unroll
        for (int u = 0; u < CH; ++u) ev[u][0] = ev[u][1] = ev[u][2] = ev[u][3] = od[u][0] = od[u][1] = od[u][2] = od[u][3] = 0.f;
        for (int r = 0; r < JE; ++r) {
            const float w = kp.tie32[size_t(r) * JE + a];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int c = half * CH + u;
                const float2 y = Ci[c * NP + 2 * r], yp = Vi[c * NP + 2 * r];
                ev[u][0] = fmaf(w, y.x, ev[u][0]);
                ev[u][1] = fmaf(w, y.y, ev[u][1]);
                ev[u][2] = fmaf(w, yp.x, ev[u][2]);
                ev[u][3] = fmaf(w, yp.y, ev[u][3]);
            }
        }
        for (int r = 0; r < JO; ++r) {
            const float w = kp.tio32[size_t(r) * JE + a];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int c = half * CH + u;
                const float2 y = Ci[c * NP + 2 * r + 1], yp = Vi[c * NP + 2 * r + 1];
                od[u][0] = fmaf(w, y.x, od[u][0]);
                od[u][1] = fmaf(w, y.y, od[u][1]);
                od[u][2] = fmaf(w, yp.x, od[u][2]);
                od[u][3] = fmaf(w, yp.y, od[u][3]);
            }
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
        const int c = half * CH + u, col = col0 + c;
        if (col >= M) continue;
        const float ex = ev[u][0], ey = ev[u][1], dex = ev[u][2], dey = ev[u][3];
        const float ox = od[u][0], oy = od[u][1], dox = od[u][2], doy = od[u][3];
        const float sz = kp.f.sz;
        for (int side = 0; side < 2; ++side) {
            const int j = side ? m - a : a;
            if (side && j == a) break;
            const float sg = side ? -1.f : 1.f;
            float2 ps = make_float2(ex + sg * ox, ey + sg * oy);
            float2 dps = make_float2((dex + sg * dox) * sz, (dey + sg * doy) * sz);
            const float z = kp.zn32[j];
            if (s_corr[c] && z >= -HEf && z <= Hf + HEf) {
                const float k = s_k[c], ekH = s_ekH[c], iden = s_iden[c];
                const float e1 = expf(-k * z), e3 = expf(k * (z - Hf));
                const float e2 = e3 * ekH, e4 = e1 * ekH;
                const float2 P = s_P[c], Q = s_Q[c];
                const float2 val = cscale(cadd(cscale(P, -(e1 - Gt * e2)), cscale(Q, e3 - Gb * e4)), iden);
                const float2 der = cscale(cadd(cscale(P, e1 + Gt * e2), cscale(Q, e3 + Gb * e4)), k * iden);
                ps = cadd(ps, val);
                dps = cadd(dps, der);
            }
            if (col == 0) {
                ps.x += Ai * z;
                dps.x += Ai;
            }
            sp[size_t(j) * M + col] = ps;
            sp[size_t(N + j) * M + col] = dps;
        }
        }
    }
    if (tid == 0) {
        double g = 0.0;
        for (int c = 0; c < CB; ++c) g += s_gauge[c];
        kp.part_gauge_far[bid] = g;
    }
}
template <int CB>
__global__ void __launch_bounds__(32 * CB, 32 / CB) k_column_mixed(KP kp) { column_mixed_body<CB>(kp, blockIdx.x); }
__global__ void __launch_bounds__(kColThreadsM, 4) k_column_mixed_batch(const __grid_constant__ ColBatch b) {
    const int s = batch_system(b.starts, b.nsys, blockIdx.x);
    column_mixed_body<kColBlockM>(b.kp[s], blockIdx.x - b.starts[s]);
}

// ---------------------------------------------------------------------------
// z transforms on the tensor cores (zgemm.cuh), mixed precision, Nz <= 256:
// k_zgemm_fwd turns the node values of both densities (planes 0, 1 of the
// spectrum) into Chebyshev coefficients in place; k_column_mixed<true> solves
// the BVPs on them; k_zgemm_inv turns the coefficients of psi_i and
// dpsi_i/dz back into node values, adding in its epilogue the factor 2/Hbar
// of the derivative, the correction of Eq. (inphisc) at the node
// (normalised form, float) and the k = 0 linear term A_i z (Sec. 5.2.2
// steps 4-6).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kZThreads, 1) k_zgemm_fwd(KP kp) {
    float* base = static_cast<float*>(kp.spec);
    const size_t ld = 2 * size_t(kp.ny) * kp.nxh, pstride = size_t(kp.nz) * ld;
    auto prep = [](int, int) {};
    auto epi = [](int, int, int, float*, int) {};
    // plane 1 (rho_o) only when the column kernel does not form its
    // coefficients from its node pairs
    zgemm_run<true>(kp.zimg_fwd, base, kp.o_pairs > 0 ? 1 : 2, pstride, kp.nz, int(ld), ld, kp.status, prep, epi, (kp.nz + kZBlock - 1) / kZBlock,
              kp.zspin, kp.node_mask);
}

// rho_o's Chebyshev coefficients (Sec. 5.2.2 step 3, the DCT-I form of the
// extrema grid) from its node values at the o_pairs node pairs (a, m - a) it
// can reach, in place in plane 1 of the spectra: the other nodes are zero,
// so each coefficient is a sum over those pairs only, S = v_a + v_{m-a} for
// even n and D = v_a - v_{m-a} for odd n (cos(pi n (m - a)/m) = (-1)^n
// cos(pi n a/m)). One block per kOcCols columns: the pairs' values of its
// columns are read first, then every coefficient row of its columns written.
constexpr int kOcCols = 64;
__global__ void __launch_bounds__(256) k_o_coeffs(KP kp) {
    __shared__ float4 sSD[kMaxOPairs][kOcCols];
    const int N = kp.nz, M = kp.ny * kp.nxh, P = kp.o_pairs, m = N - 1;
    const int col0 = blockIdx.x * kOcCols, tid = threadIdx.x;
    float2* const sp = static_cast<float2*>(kp.spec) + size_t(N) * M;   // plane 1
    for (int t = tid; t < P * kOcCols; t += blockDim.x) {
        const int q = t / kOcCols, c = t - q * kOcCols, col = col0 + c, a = kp.o_pair[q];
        float2 va = make_float2(0.f, 0.f), vb = va;
        if (col < M) {
            va = sp[size_t(a) * M + col];
            if (m - a != a) vb = sp[size_t(m - a) * M + col];
        }
        sSD[q][c] = make_float4(va.x + vb.x, va.y + vb.y, va.x - vb.x, va.y - vb.y);
    }
    __syncthreads();
    // thread: column c, coefficients n0 .. n0 + 7 for n0 = 8 (g + 4 k); the
    // warp's lanes are 32 columns sharing n0, so the transform entries are
    // one broadcast load per 4 and each column's S, D one load per pair
    const int c = tid % kOcCols, g = tid / kOcCols, col = col0 + c;
    if (col < M) {
        for (int n0 = 8 * g; n0 < N; n0 += 8 * (256 / kOcCols)) {
            float2 acc[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i] = make_float2(0.f, 0.f);
            for (int q = 0; q < P; ++q) {
                const float4 wa = __ldg(reinterpret_cast<const float4*>(kp.o_fwd + size_t(q) * N + n0));
                const float4 wb = __ldg(reinterpret_cast<const float4*>(kp.o_fwd + size_t(q) * N + n0 + 4));
                const float4 v = sSD[q][c];
                const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                for (int i = 0; i < 8; i += 2) {   // even n: S, odd n: D
                    acc[i].x = fmaf(w[i], v.x, acc[i].x);
                    acc[i].y = fmaf(w[i], v.y, acc[i].y);
                    acc[i + 1].x = fmaf(w[i + 1], v.z, acc[i + 1].x);
                    acc[i + 1].y = fmaf(w[i + 1], v.w, acc[i + 1].y);
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) sp[size_t(n0 + i) * M + col] = acc[i];
        }
    }
}

// 2^x by the PTX base-2 exponential (ex2.approx.ftz.f32)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kZThreads, 1) k_zgemm_inv(KP kp) {
    float* base = static_cast<float*>(kp.spec);
    const size_t ld = 2 * size_t(kp.ny) * kp.nxh, pstride = size_t(kp.nz) * ld;
    const float Gb = kp.f.Gb, Gt = kp.f.Gt, H = kp.f.H, HE = kp.f.HE, sz = kp.f.sz;
    const float Ai = float(kp.scal[1]);
    // the tile's 64 modes' correction, staged once per tile and plane as the
    // factors of e1 = e^{-kz} and e3 = e^{k(z-H)}: with f = iden (plane 0) or
    // k iden (plane 1), the correction is e1 A + e3 B, A = -/+ f (P + Gb ekH Q)
    // and B = f (Gt ekH P + Q) (the two terms of each of P and Q gathered);
    // s_kc: k, and whether the mode has a correction
    __shared__ float4 s_ab[kZN / 2];        // (A.re, A.im, B.re, B.im)
    __shared__ float2 s_kc[kZN / 2];
    int s_c0 = 0;
    auto prep = [&](int plane, int c0) {
        const int i = threadIdx.x, col = c0 / 2 + i;
        if (i < kZN / 2 && col < kp.ny * kp.nxh) {
            const ColP cp = kp.colp[col];
            const float f = plane == 0 ? cp.iden : cp.k * cp.iden, sa = plane == 0 ? -f : f;
            const float2 A = make_float2(sa * (cp.P.x + Gb * cp.ekH * cp.Q.x), sa * (cp.P.y + Gb * cp.ekH * cp.Q.y));
            const float2 B = make_float2(f * (Gt * cp.ekH * cp.P.x + cp.Q.x), f * (Gt * cp.ekH * cp.P.y + cp.Q.y));
            s_ab[i] = make_float4(A.x, A.y, B.x, B.y);
            s_kc[i] = make_float2(cp.k, cp.corr ? 1.f : 0.f);
        }
        s_c0 = c0;
    };
    auto epi = [&](int plane, int row, int c0, float* v, int w) {
        const float z = kp.zn32[row];
        const bool zin = z >= -HE && z <= H + HE;
        // the exponents' row factors in base 2: e^{-kz} = 2^{k lz}
        const float lz = -z * 1.44269504088896341f, lhz = -(H - z) * 1.44269504088896341f;
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
            if (i >= w) break;
            const int col = (c0 + i) >> 1, m = col - s_c0 / 2;
            float re = v[i], im = v[i + 1];
            if (plane == 1) { re *= sz; im *= sz; }
            const float2 kc = s_kc[m];
            // a warp's lanes are rows of one column, so the test of the mode
            // is uniform over the warp (modes without a correction add
            // nothing); within a mode no branches (rows would diverge): the
            // exponents are clamped at -127 (e^{-88}), where both terms are
            // below 1e-38 of the correction's amplitude, and nodes outside
            // [-H_E, H + H_E] are masked to exactly zero
            if (kc.y != 0.f) {
                // the hardware base-2 exponential: its error grows as |x| 2^-24
                // of the result, and amplitude x e^{-x} <= 0.37 amplitude, so
                // each term is within 2e-8 of its amplitude (below FP32 rounding)
                const float e1 = zin ? ex2_approx(fmaxf(kc.x * lz, -127.f)) : 0.f;
                const float e3 = zin ? ex2_approx(fmaxf(kc.x * lhz, -127.f)) : 0.f;
                const float4 ab = s_ab[m];
                re += e1 * ab.x + e3 * ab.z;
                im += e1 * ab.y + e3 * ab.w;
            }
            if (col == 0) re += plane == 0 ? Ai * z : Ai;
            v[i] = re;
            v[i + 1] = im;
        }
    };
    zgemm_run<false>(kp.zimg_inv, base, 2, pstride, kp.nz, int(ld), ld, kp.status, prep, epi, (kp.nz + kZBlock - 1) / kZBlock,
              kp.zspin, nullptr, kp.node_mask);
}

// ---------------------------------------------------------------------------
// xy FFT, inverse: columns along y for psi, -i k_y psi and dpsi/dz, then rows
// along x packing (phi, E_x) and (E_y, E_z) as one complex FFT each
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_ffty_inv(KP kp, int TK) {
    using C = typename Prec<R>::C;
    extern __shared__ __align__(16) unsigned char smraw[];
    if (kp.node_mask && !(kp.node_mask[blockIdx.y] & 2)) return;   // a plane the interpolation never reads
    C* sm = reinterpret_cast<C*>(smraw);
    const int n = kp.ny, nxh = kp.nxh;
    C* tw = sm;
    C* A = tw + n;
    C* B = A + 3 * TK * n;
    const C* twg = twy_of<R>(kp);
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const size_t plane = size_t(n) * nxh;
    const R kys = R(kTwoPi / kp.Ly);
    C* s0 = static_cast<C*>(kp.spec) + size_t(blockIdx.y) * plane;
    C* s1 = static_cast<C*>(kp.spec) + size_t(kp.nz + blockIdx.y) * plane;
    C* sb = static_cast<C*>(kp.specB) + size_t(blockIdx.y) * plane;
    const int k0 = blockIdx.x * TK;
    for (int t = threadIdx.x; t < TK * n; t += blockDim.x) {
        const int y = t / TK, c = t - y * TK, kx = k0 + c;
        C ps, dps;
        ps.x = ps.y = dps.x = dps.y = R(0);
        if (kx < nxh) {
            ps = s0[size_t(y) * nxh + kx];
            dps = s1[size_t(y) * nxh + kx];
        }
        const int my = y < (n + 1) / 2 ? y : y - n;
        const R ky = (n % 2 == 0 && y == n / 2) ? R(0) : (sizeof(R) == sizeof(double) ? R(kTwoPi * my / kp.Ly) : kys * R(my));
        C dy;
        dy.x = ky * ps.y;                          // -i k_y psi
        dy.y = -ky * ps.x;
        A[c * n + y] = ps;
        A[(TK + c) * n + y] = dy;
        A[(2 * TK + c) * n + y] = dps;
    }
    __syncthreads();
    const C* Rr = block_fft(A, B, tw, n, 3 * TK, kp.rady, kp.nrady, +1);
    for (int t = threadIdx.x; t < TK * n; t += blockDim.x) {
        const int y = t / TK, c = t - y * TK, kx = k0 + c;
        if (kx >= nxh) continue;
        s0[size_t(y) * nxh + kx] = Rr[c * n + y];
        sb[size_t(y) * nxh + kx] = Rr[(TK + c) * n + y];
        s1[size_t(y) * nxh + kx] = Rr[(2 * TK + c) * n + y];
    }
}

template <class R>
__global__ void k_fftx_inv(KP kp, int P) {
    using C = typename Prec<R>::C;
    using V4 = typename Prec<R>::V4;
    extern __shared__ __align__(16) unsigned char smraw[];
    C* sm = reinterpret_cast<C*>(smraw);
    const int n = kp.nx, nxh = kp.nxh;
    C* tw = sm;
    C* A = tw + n;
    C* B = A + 2 * P * n;
    const C* twg = twx_of<R>(kp);
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const C* spec = static_cast<const C*>(kp.spec);
    const C* specB = static_cast<const C*>(kp.specB);
    V4* fields = static_cast<V4*>(kp.fields);
    const int nrows = kp.nz * kp.ny;
    const size_t S = size_t(nrows) * nxh;
    const R kxs = R(kTwoPi / kp.Lx);
    const int r0 = blockIdx.x * P;
    // rows past the grid or at nodes the interpolation never reads
    const unsigned long long skip = f_rows_skip(kp, r0, P, nrows);
    if (skip == (P >= 64 ? ~0ull : (1ull << P) - 1ull)) return;
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t / n, k = t - p * n, row = r0 + p;
        C z1, z2;
        z1.x = z1.y = z2.x = z2.y = R(0);
        if (!((skip >> p) & 1ull)) {
            const bool hi = k >= nxh;
            const int kk = hi ? n - k : k;
            C a = spec[size_t(row) * nxh + kk];
            C b = specB[size_t(row) * nxh + kk];
            C c = spec[S + size_t(row) * nxh + kk];
            const bool edge = kk == 0 || (n % 2 == 0 && kk == n / 2);
            if (edge) { a.y = R(0); b.y = R(0); c.y = R(0); }
            const R kxd = edge ? R(0) : (sizeof(R) == sizeof(double) ? R(kTwoPi * kk / kp.Lx) : kxs * R(kk));
            C r, mc;
            r.x = kxd * a.y;                     // -i k_x psi
            r.y = -kxd * a.x;
            mc.x = -c.x;                         // E_z = -dpsi/dz
            mc.y = -c.y;
            if (hi) { a = cconj(a); r = cconj(r); b = cconj(b); mc = cconj(mc); }
            z1.x = a.x - r.y;                    // phi + i E_x
            z1.y = a.y + r.x;
            z2.x = b.x - mc.y;                   // E_y + i E_z
            z2.y = b.y + mc.x;
        }
        A[(2 * p) * n + k] = z1;
        A[(2 * p + 1) * n + k] = z2;
    }
    __syncthreads();
    const C* Rr = block_fft(A, B, tw, n, 2 * P, kp.radx, kp.nradx, +1);
    const R s = R(kp.inv_nxny);
    for (int t = threadIdx.x; t < P * n; t += blockDim.x) {
        const int p = t / n, x = t - p * n, row = r0 + p;
        if ((skip >> p) & 1ull) continue;
        const C u = Rr[(2 * p) * n + x], v = Rr[(2 * p + 1) * n + x];
        fields[size_t(row) * n + x] = Prec<R>::v4(u.x * s, u.y * s, v.x * s, v.y * s);
    }
}

// ---------------------------------------------------------------------------
// interpolation, Sec. 5.2.2 step 7: one warp per charge, grid quadrature of
// the kernel times the four fields (lane sums in R, warp sum in double)
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_interp(KP kp) {
    using V4 = typename Prec<R>::V4;
    extern __shared__ __align__(16) unsigned char smraw[];
    R* smi = reinterpret_cast<R*>(smraw);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    R* wx = smi + w * (2 * kMaxSupport + kMaxNz);
    R* wy = wx + kMaxSupport;
    R* wzz = wy + kMaxSupport;
    const int slot = blockIdx.x * (blockDim.x >> 5) + w;
    if (slot >= kp.n) return;
    // charges in cell-list order when there is one: neighbouring warps then
    // gather overlapping parts of the grid, which stay in L2
    const int k = kp.near_on ? kp.sorted_idx[slot] : slot;
    const V4* fields = static_cast<const V4*>(kp.fields);
    const double4_32a p = kp.near_on ? kp.sorted[slot] : kp.part[k];
    const double x = p.x, y = p.y, z = p.z, HE = kp.HE;
    const int ix0 = int(ceil((x - HE) / kp.hx)), ix1 = int(floor((x + HE) / kp.hx));
    const int iy0 = int(ceil((y - HE) / kp.hy)), iy1 = int(floor((y + HE) / kp.hy));
    const int sx = ix1 - ix0 + 1, sy = iy1 - iy0 + 1;
    int j0 = kp.nz, j1 = -1;
    for (int j = lane; j < kp.nz; j += 32) {
        if (fabs(kp.zn[j] - z) <= HE) { j0 = min(j0, j); j1 = max(j1, j); }
    }
    for (int o = 16; o > 0; o >>= 1) {
        j0 = min(j0, __shfl_xor_sync(0xffffffffu, j0, o));
        j1 = max(j1, __shfl_xor_sync(0xffffffffu, j1, o));
    }
    const int sz = j1 - j0 + 1;
    const R ig2 = R(1.0 / (2.0 * kp.gt * kp.gt));
    const R s1 = R(kp.s1norm);
    // offsets: base in double, then d0 + i h in R
    const R d0x = R(double(ix0) * kp.hx - x), d0y = R(double(iy0) * kp.hy - y);
    for (int i = lane; i < sx; i += 32) {
        const R d = d0x + R(i) * R(kp.hx);
        wx[i] = s1 * dexp(-d * d * ig2);
    }
    for (int i = lane; i < sy; i += 32) {
        const R d = d0y + R(i) * R(kp.hy);
        wy[i] = s1 * dexp(-d * d * ig2);
    }
    for (int i = lane; i < sz; i += 32) {
        const R d = R(kp.zn[j0 + i] - z);
        wzz[i] = R(kp.wz[j0 + i]) * (s1 * dexp(-d * d * ig2));
    }
    __syncwarp();
    const R wxy = R(kp.hx * kp.hy);
    R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const int sxy = sx * sy;
    for (int t = lane; t < sz * sxy; t += 32) {
        const int jz = t / sxy, r = t - jz * sxy, iy = r / sx, ix = r - iy * sx;
        const R wt = wxy * wzz[jz] * wy[iy] * wx[ix];
        const size_t g = (size_t(j0 + jz) * kp.ny + wrap_index(iy0 + iy, kp.ny)) * kp.nx + wrap_index(ix0 + ix, kp.nx);
        const V4 f = fields[g];
        a0 = fma(wt, f.x, a0);
        a1 = fma(wt, f.y, a1);
        a2 = fma(wt, f.z, a2);
        a3 = fma(wt, f.w, a3);
    }
    double b0, b1, b2, b3;
    if (sizeof(R) == sizeof(float)) {
        b0 = warp_sum_f(float(a0)); b1 = warp_sum_f(float(a1)); b2 = warp_sum_f(float(a2)); b3 = warp_sum_f(float(a3));
    } else {
        b0 = warp_sum(double(a0)); b1 = warp_sum(double(a1)); b2 = warp_sum(double(a2)); b3 = warp_sum(double(a3));
    }
    if (lane == 0) kp.far[k] = make_double4_32a(b0, b1, b2, b3);
}

// Mixed precision: one warp per charge, on the window k_sources_f stored for
// it (the support of the charge's own source). Each lane takes (x, y)
// columns of the support and walks down z with one pointer step per node,
// all in float; node distances use z and z_j as float pairs (~1e-7).
__global__ void __launch_bounds__(32 * kMaxInterpWarps) k_interp_f32(KP kp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float* smi = reinterpret_cast<float*>(smraw);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* wx = smi + w * (2 * kMaxSupport + kMaxNz);
    float* wy = wx + kMaxSupport;
    float* wzz = wy + kMaxSupport;
    const int slot = blockIdx.x * (blockDim.x >> 5) + w;
    if (slot >= kp.n) return;
    const int k = kp.near_on ? kp.sorted_idx[slot] : slot;
    const IRec r = kp.irec[slot];
    const int sx = r.sx, sy = r.sy, j0 = r.j0, sz = r.j1 - r.j0 + 1;
    const float ig2 = kp.f.ig2, s1 = kp.f.s1norm;
    for (int i = lane; i < sx; i += 32) {
        const float d = r.d0x + float(i) * kp.f.hx;
        wx[i] = s1 * expf(-d * d * ig2);
    }
    for (int i = lane; i < sy; i += 32) {
        const float d = r.d0y + float(i) * kp.f.hy;
        wy[i] = s1 * expf(-d * d * ig2);
    }
    for (int i = lane; i < sz; i += 32) {
        const int j = j0 + i;
        const float d = (kp.zn32[j] - r.zhi) + (kp.znlo32[j] - r.zlo);
        wzz[i] = kp.wzh32[j] * (s1 * expf(-d * d * ig2));
    }
    __syncwarp();
    const float4* fields = static_cast<const float4*>(kp.fields);
    const int nx = kp.nx, ny = kp.ny;
    const size_t plane = size_t(ny) * nx;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    // column t = lane + 32 i of the sx x sy support, as (ix, iy), advanced
    // incrementally; the support fits the grid, so one wrap suffices
    int iy = lane / max(sx, 1), ix = lane - iy * sx;
    const int xw = wrap_index(r.xlo, nx), yw = wrap_index(r.ylo, ny);
    for (; sx > 0 && iy < sy; ix += 32) {
        while (ix >= sx) { ix -= sx; ++iy; }
        if (iy >= sy) break;
        int gx = xw + ix, gy = yw + iy;
        if (gx >= nx) gx -= nx;
        if (gy >= ny) gy -= ny;
        const float wxy = wx[ix] * wy[iy];
        const float4* f = fields + (size_t(j0) * ny + gy) * nx + gx;
        for (int jz = 0; jz < sz; ++jz, f += plane) {
            const float4 v = __ldg(f);
            const float wt = wxy * wzz[jz];
            a0 = fmaf(wt, v.x, a0);
            a1 = fmaf(wt, v.y, a1);
            a2 = fmaf(wt, v.z, a2);
            a3 = fmaf(wt, v.w, a3);
        }
    }
    a0 = warp_sum_f(a0);
    a1 = warp_sum_f(a1);
    a2 = warp_sum_f(a2);
    a3 = warp_sum_f(a3);
    if (lane < 4) {
        const float v = lane == 0 ? a0 : lane == 1 ? a1 : lane == 2 ? a2 : a3;
        reinterpret_cast<double*>(kp.far + k)[lane] = double(v);
    }
}

// ---------------------------------------------------------------------------
// near field over a cell list (Sec. 4.2): counting sort, then one thread per
// charge over the neighbouring cells, with one image per wall
// ---------------------------------------------------------------------------
__global__ void k_scan_cells(KP kp) {
    __shared__ int sums[1024];
    const int n = kp.ncells, tid = threadIdx.x, bs = blockDim.x;
    const int chunk = (n + bs - 1) / bs;
    const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += kp.cell_count[i];
    sums[tid] = s;
    __syncthreads();
    for (int o = 1; o < bs; o <<= 1) {
        const int v = tid >= o ? sums[tid - o] : 0;
        __syncthreads();
        sums[tid] += v;
        __syncthreads();
    }
    int run = sums[tid] - s;
    for (int i = lo; i < hi; ++i) {
        kp.cell_start[i] = run;
        run += kp.cell_count[i];
    }
    if (tid == bs - 1) kp.cell_start[n] = sums[bs - 1];
}

__global__ void k_scatter_cells(KP kp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kp.n) return;
    const int c = kp.cell_of[k];
    const int slot = kp.cell_start[c] + atomicAdd(&kp.cell_fill[c], 1);
    const double4_32a p = kp.part[k];
    kp.sorted[slot] = p;
    kp.sorted_idx[slot] = k;
    const int cz = c % kp.ncz, cx = (c / kp.ncz) % kp.ncx, cy = c / (kp.ncz * kp.ncx);
    kp.sorted_rel[slot] = make_float4(float(p.x - cx * kp.cwx), float(p.y - cy * kp.cwy), float(p.z - cz * kp.cwz),
                                      float(p.w));
}

template <class R>
__device__ __forceinline__ void near_cell(const KP& kp, int cell, double x, double y, double zt, double zsign,
                                          double zoff, double strength, double rc2,
                                          R& phi, R& ex, R& ey, R& ez) {
    const int s0 = kp.cell_start[cell], s1 = kp.cell_start[cell + 1];
    for (int s = s0; s < s1; ++s) {
        const double4_32a src = kp.sorted[s];
        const double dx = min_image(x - src.x, kp.Lx);
        const double dy = min_image(y - src.y, kp.Ly);
        const double dz = zt - (zoff + zsign * src.z);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < rc2) {
            R g, d;
            if (sizeof(R) == sizeof(float) && kp.near_quad) {
                float gf, df;
                near_kernel_quad(kp, float(sqrt(r2)), gf, df);
                g = R(gf);
                d = R(df);
            } else {
                near_kernel<R>(R(sqrt(r2)), R(kp.na1), R(kp.na2), R(kp.gw), R(kp.eps), g, d);
            }
            const R qs = R(strength * src.w);
            phi += qs * g;
            ex -= qs * d * R(dx);
            ey -= qs * d * R(dy);
            ez -= qs * d * R(dz);
        }
    }
}

template <class R>
__global__ void k_near(KP kp) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= kp.n) return;
    const double4_32a t = kp.sorted[s];
    const double x = t.x, y = t.y, z = t.z;
    const int cx = min(kp.ncx - 1, max(0, int(x / kp.cwx)));
    const int cy = min(kp.ncy - 1, max(0, int(y / kp.cwy)));
    const int cz = min(kp.ncz - 1, max(0, int(z / kp.cwz)));
    const double rc2 = kp.r_cut * kp.r_cut;
    R phi = 0, ex = 0, ey = 0, ez = 0;
    const int nxc = kp.ncx >= 3 ? 3 : kp.ncx, nyc = kp.ncy >= 3 ? 3 : kp.ncy;
    // pass 0: charges; pass 1: images below z = 0; pass 2: images above z = H
    for (int pass = 0; pass < 3; ++pass) {
        int zl, zh;
        double zsign, zoff, st;
        if (pass == 0) { zl = max(0, cz - 1); zh = min(kp.ncz - 1, cz + 1); zsign = 1.0; zoff = 0.0; st = 1.0; }
        else if (pass == 1) {
            if (!(z < kp.r_cut) || kp.Gb == 0.0) continue;
            zl = zh = 0; zsign = -1.0; zoff = 0.0; st = -kp.Gb;
        } else {
            if (!(kp.H - z < kp.r_cut) || kp.Gt == 0.0) continue;
            zl = zh = kp.ncz - 1; zsign = -1.0; zoff = 2.0 * kp.H; st = -kp.Gt;
        }
        for (int zc = zl; zc <= zh; ++zc) {
            for (int oy = 0; oy < nyc; ++oy) {
                const int yc = kp.ncy >= 3 ? wrap_index(cy - 1 + oy, kp.ncy) : oy;
                for (int ox = 0; ox < nxc; ++ox) {
                    const int xc = kp.ncx >= 3 ? wrap_index(cx - 1 + ox, kp.ncx) : ox;
                    near_cell<R>(kp, cell_index(kp, xc, yc, zc), x, y, z, zsign, zoff, st, rc2, phi, ex, ey, ez);
                }
            }
        }
    }
    kp.nearv[kp.sorted_idx[s]] = make_double4_32a(phi, ex, ey, ez);
}

// Near field in float (mixed precision): positions are kept as float offsets
// from their cell's corner, so a pair's separation is the offset difference
// plus a whole number of cell widths; no double arithmetic per pair. Images:
// the bottom image of a source in cell layer 0 sits at -z, so the z
// separation from a target in layer 0 is z_t + z_s; for the top image use the
// distances to z = H, which are (cell height - offset) in the top layer.
__global__ void k_near_f32(KP kp) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= kp.n) return;
    const float4 t = kp.sorted_rel[s];
    const double4_32a ta = kp.sorted[s];
    const int cx = min(kp.ncx - 1, max(0, int(ta.x / kp.cwx)));
    const int cy = min(kp.ncy - 1, max(0, int(ta.y / kp.cwy)));
    const int cz = min(kp.ncz - 1, max(0, int(ta.z / kp.cwz)));
    const float cwx = float(kp.cwx), cwy = float(kp.cwy), cwz = float(kp.cwz);
    const float Lx = float(kp.Lx), Ly = float(kp.Ly);
    const float rc2 = float(kp.r_cut * kp.r_cut);
    const bool wrap3x = kp.ncx >= 3, wrap3y = kp.ncy >= 3;
    const int nxc = wrap3x ? 3 : kp.ncx, nyc = wrap3y ? 3 : kp.ncy;
    // the neighbour columns and rows (wrapped once: the unwrapped index lies
    // in [-1, n]) and the shifts of their cell-relative offsets, once
    int xcs[3], ycs[3];
    float sxhs[3], syhs[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        const int xu = wrap3x ? cx - 1 + o : o, yu = wrap3y ? cy - 1 + o : o;
        xcs[o] = xu < 0 ? xu + kp.ncx : (xu >= kp.ncx ? xu - kp.ncx : xu);
        ycs[o] = yu < 0 ? yu + kp.ncy : (yu >= kp.ncy ? yu - kp.ncy : yu);
        sxhs[o] = float(cx - xu) * cwx;
        syhs[o] = float(cy - yu) * cwy;
    }
    float phi = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
    auto pair = [&](float dx, float dy, float dz, float qs) {
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < rc2) {
            float g, d;
            if (kp.near_quad) near_kernel_quad(kp, sqrtf(r2), g, d);
            else near_kernel<float>(sqrtf(r2), float(kp.na1), float(kp.na2), float(kp.gw), float(kp.eps), g, d);
            phi += qs * g;
            ex -= qs * d * dx;
            ey -= qs * d * dy;
            ez -= qs * d * dz;
        }
    };
    for (int pass = 0; pass < 3; ++pass) {
        int zl, zh;
        float st;
        if (pass == 0) { zl = max(0, cz - 1); zh = min(kp.ncz - 1, cz + 1); st = 1.f; }
        else if (pass == 1) {
            if (!(ta.z < kp.r_cut) || kp.Gb == 0.0) continue;
            zl = zh = 0; st = float(-kp.Gb);
        } else {
            if (!(kp.H - ta.z < kp.r_cut) || kp.Gt == 0.0) continue;
            zl = zh = kp.ncz - 1; st = float(-kp.Gt);
        }
        for (int zc = zl; zc <= zh; ++zc) {
            for (int oy = 0; oy < nyc; ++oy) {
                const int yc = ycs[oy];
                const float syh = syhs[oy];
                for (int ox = 0; ox < nxc; ++ox) {
                    const int xc = xcs[ox];
                    const int cell = cell_index(kp, xc, yc, zc);
                    const float sxh = sxhs[ox];
                    for (int q = kp.cell_start[cell]; q < kp.cell_start[cell + 1]; ++q) {
                        const float4 src = kp.sorted_rel[q];
                        float dx = t.x - src.x + sxh, dy = t.y - src.y + syh;
                        if (!wrap3x) { if (dx > 0.5f * Lx) dx -= Lx; else if (dx < -0.5f * Lx) dx += Lx; }
                        if (!wrap3y) { if (dy > 0.5f * Ly) dy -= Ly; else if (dy < -0.5f * Ly) dy += Ly; }
                        float dz;
                        if (pass == 0) dz = t.z - src.z + float(cz - zc) * cwz;
                        else if (pass == 1) dz = t.z + src.z;
                        else dz = -((cwz - t.z) + (cwz - src.z));
                        pair(dx, dy, dz, st * src.w);
                    }
                }
            }
        }
    }
    kp.nearv[kp.sorted_idx[s]] = make_double4_32a(phi, ex, ey, ez);
}

// Integral over a wall plane of the pointwise near-field kernel Eq. (Gnear)
// of a unit charge at distance d from it, truncated at r_cut like the near
// field: (1/(2 eps)) int_d^{r_cut} [erf(r/a1) - erf(r/a2)] dr, written with
// I(x, a) = int_x^inf erfc(r/a) dr = a (e^{-(x/a)^2}/sqrt(pi) - (x/a) erfc(x/a)).
__device__ double wall_near_planar(double d, const KP& kp) {
    d = fabs(d);
    if (d >= kp.r_cut) return 0.0;
    auto I = [](double x, double a) {
        const double u = x / a;
        return a * (exp(-u * u) * 0.56418958354775628695 - u * erfc(u));
    };
    const double a1 = kp.pa1, a2 = kp.pa2, rc = kp.r_cut;
    return ((I(d, a2) - I(d, a1)) - (I(rc, a2) - I(rc, a1))) / (2.0 * kp.eps);
}

// pointwise near-field potential at the origin (gauge of Sec. 5.2.2); with
// wall charges also the per-charge terms of their energy: q phibar_sigma and
// the near field's planar integrals at z = 0 and z = H (charge and one image
// per wall, the near field's sources)
__global__ void k_origin(KP kp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (kp.sigma_on) {
        double c = 0.0, n0 = 0.0, nH = 0.0;
        if (k < kp.n) {
            const double4_32a p = kp.part[k];
            const double q = p.w, z = p.z, H = kp.H;
            c = q * kp.wall_phi[k];
            if (kp.near_on) {
                n0 = q * ((1.0 - kp.Gb) * wall_near_planar(z, kp) - kp.Gt * wall_near_planar(2.0 * H - z, kp));
                nH = q * ((1.0 - kp.Gt) * wall_near_planar(H - z, kp) - kp.Gb * wall_near_planar(H + z, kp));
            }
        }
        c = block_sum(c);
        n0 = block_sum(n0);
        nH = block_sum(nH);
        if (threadIdx.x == 0) {
            const int nb = kp.n_charge_blocks;
            kp.part_wall[blockIdx.x] = c;
            kp.part_wall[nb + blockIdx.x] = n0;
            kp.part_wall[2 * nb + blockIdx.x] = nH;
        }
    }
    double v = 0.0;
    const double4_32a p = k < kp.n ? kp.part[k] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
    // x, y lie in [0, L]: the periodic distance to the origin is min(x, L - x),
    // and a charge farther than r_cut in x or y reaches it with neither
    // itself nor an image (the margin covers the rounding of min_image)
    const double lim = kp.r_cut * (1.0 + 1e-9);
    const bool cand = k < kp.n && fmin(p.x, kp.Lx - p.x) <= lim && fmin(p.y, kp.Ly - p.y) <= lim;
    if (cand && kp.near_on) {
        const double dx = min_image(0.0 - p.x, kp.Lx), dy = min_image(0.0 - p.y, kp.Ly);
        const double rc = kp.r_cut;
        const double r = sqrt(dx * dx + dy * dy + p.z * p.z);
        const double zt = 2.0 * kp.H - p.z;
        const double rt = sqrt(dx * dx + dy * dy + zt * zt);
        double g, d;
        if (r < rc) {
            near_kernel<double>(r, kp.pa1, kp.pa2, kp.gw, kp.eps, g, d);
            v += p.w * g;                 // the charge
            v += -kp.Gb * p.w * g;        // its image below z = 0 (same distance)
        }
        if (rt < rc) {
            near_kernel<double>(rt, kp.pa1, kp.pa2, kp.gw, kp.eps, g, d);
            v += -kp.Gt * p.w * g;
        }
    }
    const double s = block_sum(v);
    if (threadIdx.x == 0) kp.part_gauge_near[blockIdx.x] = s;
}

// ---------------------------------------------------------------------------
// gauge constant, assembly, energy
// ---------------------------------------------------------------------------
__global__ void k_final_gauge(KP kp) {
    double f = 0.0, nn = 0.0, q1 = 0.0, q2 = 0.0;
    for (int i = threadIdx.x; i < kp.n_col_blocks; i += blockDim.x) f += kp.part_gauge_far[i];
    for (int i = threadIdx.x; i < kp.n_charge_blocks; i += blockDim.x) {
        nn += kp.part_gauge_near[i];
        q1 += kp.part_q[i];
        q2 += kp.part_q[kp.n_charge_blocks + i];
    }
    f = block_sum(f);
    nn = block_sum(nn);
    q1 = block_sum(q1);
    q2 = block_sum(q2);
    if (threadIdx.x == 0) {
        const double phi_f0 = f * kp.inv_nxny;
        kp.scal[0] = -(phi_f0 + nn);
        kp.scal[2] = phi_f0;
        kp.scal[3] = nn;
        kp.scal[5] = q1;
        kp.scal[6] = q2;
    }
}

__global__ void k_assemble(KP kp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double u = 0.0;
    if (k < kp.n) {
        const double B = kp.scal[0];
        const double4_32a f = kp.far[k];
        const double4_32a nn = kp.near_on ? kp.nearv[k] : make_double4_32a(0, 0, 0, 0);
        const double q = kp.part[k].w;
        const double phi = f.x + nn.x + B;
        if (kp.out_phi) kp.out_phi[k] = phi;
        if (kp.out_force) {
            kp.out_force[3 * k] = q * (f.y + nn.y);
            kp.out_force[3 * k + 1] = q * (f.z + nn.z);
            kp.out_force[3 * k + 2] = q * (f.w + nn.w);
        }
        u = q * phi;
    }
    const double s = block_sum(u);
    if (threadIdx.x == 0) kp.part_u[blockIdx.x] = s;
}

// U = 1/2 sum q phibar (Eq. (Ufinal)); with wall charges plus the wall term
// 1/2 int (sigma_b phi(x, y, 0) + sigma_t phi(x, y, H)): for k = 0 the total
// wall charge times the plane-averaged pointwise potential at the wall (far
// part from the k = 0 column, near part from the planar sums, gauge B), for
// k != 0 by Green's reciprocity 1/2 sum q phibar_sigma plus the wall charges'
// own term fixed when they were set
__global__ void k_final_energy(KP kp) {
    const int nb = kp.n_charge_blocks;
    double u = 0.0, c = 0.0, n0 = 0.0, nH = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        u += kp.part_u[i];
        if (kp.sigma_on) {
            c += kp.part_wall[i];
            n0 += kp.part_wall[nb + i];
            nH += kp.part_wall[2 * nb + i];
        }
    }
    u = block_sum(u);
    if (kp.sigma_on) {
        c = block_sum(c);
        n0 = block_sum(n0);
        nH = block_sum(nH);
    }
    if (threadIdx.x == 0) {
        double U = 0.5 * u;
        if (kp.sigma_on) {
            const double B = kp.scal[0], area = kp.Lx * kp.Ly;
            const double phi0 = kp.scal[7] * kp.inv_nxny + B + n0 / area;
            const double phiH = kp.scal[8] * kp.inv_nxny + B + nH / area;
            U += 0.5 * (kp.sig_Qb * phi0 + kp.sig_Qt * phiH) + 0.5 * c + kp.sig_self;
        }
        kp.scal[4] = U;
    }
}

// ---------------------------------------------------------------------------
// wall charges: set-up kernels (run once per dpslab_plan_set_wall_charge) and
// the per-solve gather of their correction at the charges
// ---------------------------------------------------------------------------
// sigma_b into plane 0 and sigma_t into plane 1 of rho_i (the rest zeroed
// before), for the forward xy transform
template <class R>
__global__ void k_wall_fill(KP kp, const double* sig) {
    const size_t plane = size_t(kp.ny) * kp.nx;
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < 2 * plane) static_cast<R*>(kp.rho)[i] = R(sig[i]);
}

// the two transformed planes -> sig_hat (double)
template <class R>
__global__ void k_wall_hat(KP kp, double2* hat) {
    using C = typename Prec<R>::C;
    const int M = kp.ny * kp.nxh;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * M) {
        const C v = static_cast<const C*>(kp.spec)[i];
        hat[i] = make_double2(double(v.x), double(v.y));
    }
}

// node values of the wall charges' own correction (Eq. (inphisc) with
// m_phi = 0, m_E = +sigma_b, -sigma_t) for 0 < k <= pi/h at nodes in
// [-H_E, H + H_E], zero elsewhere, and zero derivative planes, laid out as
// the inverse transforms read psi and dpsi/dz
template <class R>
__global__ void k_wall_nodes(KP kp, const double2* hat) {
    using C = typename Prec<R>::C;
    const int M = kp.ny * kp.nxh;
    const size_t S = size_t(kp.nz) * M;
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= S) return;
    const int j = int(i / M), col = int(i - size_t(j) * M);
    C* spec = static_cast<C*>(kp.spec);
    C zero;
    zero.x = zero.y = R(0);
    spec[S + i] = zero;
    const int iy = col / kp.nxh, ix = col - iy * kp.nxh;
    const int my = iy < (kp.ny + 1) / 2 ? iy : iy - kp.ny;
    const double kx = kTwoPi * ix / kp.Lx, ky = kTwoPi * my / kp.Ly;
    const double k = sqrt(kx * kx + ky * ky), z = kp.zn[j];
    C out = zero;
    if (k > 0.0 && k <= kp.kmax && z >= -kp.HE && z <= kp.H + kp.HE) {
        const double ie = 1.0 / (kp.eps * k);
        const double2 P = cscale(hat[col], -kp.db * ie);
        const double2 Q = cscale(hat[M + col], kp.dt * ie);
        const double ekH = exp(-k * kp.H);
        const double den = 1.0 - kp.Gb * kp.Gt * ekH * ekH;
        const double e1 = exp(-k * z), e2 = exp(k * (z - 2.0 * kp.H)), e3 = exp(k * (z - kp.H)), e4 = exp(-k * (z + kp.H));
        const double2 v = cscale(cadd(cscale(P, -(e1 - kp.Gt * e2)), cscale(Q, e3 - kp.Gb * e4)), 1.0 / den);
        out.x = R(v.x);
        out.y = R(v.y);
    }
    spec[i] = out;
}

// phi component of the inverse-transformed field grid -> sig_grid
template <class R>
__global__ void k_wall_grid(KP kp, R* grid) {
    using V4 = typename Prec<R>::V4;
    const size_t G = size_t(kp.nz) * kp.ny * kp.nx;
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < G) grid[i] = static_cast<const V4*>(kp.fields)[i].x;
}

// 1/2 int sigma phi_sigma over both walls for k != 0, by Parseval on the
// half spectrum (single block)
__global__ void k_wall_self(KP kp, const double2* hat, double* out) {
    const int M = kp.ny * kp.nxh;
    double acc = 0.0;
    for (int col = threadIdx.x; col < M; col += blockDim.x) {
        const int iy = col / kp.nxh, ix = col - iy * kp.nxh;
        const int my = iy < (kp.ny + 1) / 2 ? iy : iy - kp.ny;
        const double kx = kTwoPi * ix / kp.Lx, ky = kTwoPi * my / kp.Ly;
        const double k = sqrt(kx * kx + ky * ky);
        if (!(k > 0.0 && k <= kp.kmax)) continue;
        const double ie = 1.0 / (kp.eps * k);
        const double2 sb = hat[col], st = hat[M + col];
        const double2 P = cscale(sb, -kp.db * ie), Q = cscale(st, kp.dt * ie);
        const double ekH = exp(-k * kp.H);
        const double den = 1.0 - kp.Gb * kp.Gt * ekH * ekH;
        // correction at z = 0 and z = H
        const double2 v0 = cscale(cadd(cscale(P, -(1.0 - kp.Gt * ekH * ekH)), cscale(Q, ekH - kp.Gb * ekH)), 1.0 / den);
        const double2 vH = cscale(cadd(cscale(P, -(ekH - kp.Gt * ekH)), cscale(Q, 1.0 - kp.Gb * ekH * ekH)), 1.0 / den);
        const double mult = (ix == 0 || (kp.nx % 2 == 0 && ix == kp.nx / 2)) ? 1.0 : 2.0;
        acc += mult * (sb.x * v0.x + sb.y * v0.y + st.x * vH.x + st.y * vH.y);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = 0.5 * acc * kp.hx * kp.hy * kp.inv_nxny;
}

// phibar of the wall charges' correction at each charge: the far field's
// interpolation (Sec. 5.2.2 step 7) of one scalar grid; one warp per charge
template <class R>
__global__ void k_wall_cross(KP kp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    R* smi = reinterpret_cast<R*>(smraw);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    R* wx = smi + w * (2 * kMaxSupport + kMaxNz);
    R* wy = wx + kMaxSupport;
    R* wzz = wy + kMaxSupport;
    const int k = blockIdx.x * (blockDim.x >> 5) + w;
    if (k >= kp.n) return;
    const R* grid = static_cast<const R*>(kp.sig_grid);
    const double4_32a p = kp.part[k];
    const double x = p.x, y = p.y, z = p.z, HE = kp.HE;
    const int ix0 = int(ceil((x - HE) / kp.hx)), ix1 = int(floor((x + HE) / kp.hx));
    const int iy0 = int(ceil((y - HE) / kp.hy)), iy1 = int(floor((y + HE) / kp.hy));
    const int sx = ix1 - ix0 + 1, sy = iy1 - iy0 + 1;
    int j0 = kp.nz, j1 = -1;
    for (int j = lane; j < kp.nz; j += 32) {
        if (fabs(kp.zn[j] - z) <= HE) { j0 = min(j0, j); j1 = max(j1, j); }
    }
    for (int o = 16; o > 0; o >>= 1) {
        j0 = min(j0, __shfl_xor_sync(0xffffffffu, j0, o));
        j1 = max(j1, __shfl_xor_sync(0xffffffffu, j1, o));
    }
    const int sz = j1 - j0 + 1;
    const double ig2 = 1.0 / (2.0 * kp.gt * kp.gt);
    const double s1 = kp.s1norm;
    for (int i = lane; i < sx; i += 32) {
        const double d = double(ix0 + i) * kp.hx - x;
        wx[i] = R(s1 * exp(-d * d * ig2));
    }
    for (int i = lane; i < sy; i += 32) {
        const double d = double(iy0 + i) * kp.hy - y;
        wy[i] = R(s1 * exp(-d * d * ig2));
    }
    for (int i = lane; i < sz; i += 32) {
        const double d = kp.zn[j0 + i] - z;
        wzz[i] = R(kp.wz[j0 + i] * (s1 * exp(-d * d * ig2)));
    }
    __syncwarp();
    const R wxy = R(kp.hx * kp.hy);
    R a = 0;
    const int sxy = sx * sy;
    for (int t = lane; t < sz * sxy; t += 32) {
        const int jz = t / sxy, r = t - jz * sxy, iy = r / sx, ix = r - iy * sx;
        const size_t g = (size_t(j0 + jz) * kp.ny + wrap_index(iy0 + iy, kp.ny)) * kp.nx + wrap_index(ix0 + ix, kp.nx);
        a = fma(wxy * wzz[jz] * wy[iy] * wx[ix], grid[g], a);
    }
    const double b = warp_sum(double(a));
    if (lane == 0) kp.wall_phi[k] = b;
}

}  // namespace

// ===========================================================================
// plan
// ===========================================================================
struct dpslab_plan {
    dpslab_params p{};
    dpslab_derived d{};
    int64_t max_n = 0;
    int device = 0;
    int nxh = 0;
    size_t G = 0, S = 0;
    int px_fwd = 1, tk_fwd = 1, tk_inv = 1, px_inv = 1;
    int interp_warps = kInterpWarps;   // warps (charges) per block of the interpolation
    int col_cb = 0;                    // modes per block of the column kernel (tensor-core form: 8 W)
    int tc_r = 4;                      // tensor-core form: rows of n per lane, ceil(nz / 32)
    int spread_cpt = 1;                // x columns per thread of the mixed spreading
    int p2x = 0, p2y = 0, lognx = 0, logny = 0;        // power-of-two FFT kernels in x, y
    bool ztensor = false;                              // z transforms as tensor-core GEMMs
    int zgrid = 0;                                     // persistent CTAs of the z GEMMs
    int col_grid = 0;                                  // persistent blocks of the tensor-core form's column kernel
    int thr_x_fwd = 256, thr_x_inv = 256, thr_y_fwd = 256, thr_y_inv = 256;
    size_t sm_fftx_fwd = 0, sm_ffty_fwd = 0, sm_ffty_inv = 0, sm_fftx_inv = 0, sm_col = 0, sm_interp = 0, sm_spread = 0;
    KP kp{};
    // allocations
    void* tables = nullptr;
    void* work = nullptr;             // owned workspace (null when bound to a shared one)
    size_t work_bytes = 0;            // size of the workspace this plan needs
    size_t src_bytes = 0, scan_n = 0, rsz = 8;
    int64_t device_bytes = 0;
    double* d_pos = nullptr;    // staging for dpslab_solve_host
    double* d_q = nullptr;
    double* d_phi = nullptr;
    double* d_force = nullptr;
    double* h_scal = nullptr;   // pinned
    int* h_status = nullptr;
    int* scan_part = nullptr;     // block sums and offsets of the multi-block scans
    void* sig_mem = nullptr;      // wall charges: transforms, correction grid, scratch
    size_t sig_bytes = 0;
    cudaEvent_t done = nullptr;   // end of an enqueued (asynchronous) solve
    // the near field runs on its own stream, overlapping the far field: it
    // forks after the cell list and joins before the assembly
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool in_flight = false;
    bool bound = false;           // a workspace is bound (owned, a batch's, or the caller's)
    int64_t last_n = 0;
    int launches = 0;
    int profiling = 0;                 // 0 off, 1 stage events, 2 stage events with the near field in line
    bool near_timed = false;           // the last profiled solve timed the near field on the second stream
    cudaEvent_t ev[DPSLAB_NSTAGES + 1] = {};
    cudaEvent_t ev_near[2] = {};
    double stage_ms[DPSLAB_NSTAGES] = {};
};

namespace {

int cuda_err(cudaError_t e) {
    return e == cudaSuccess ? DPSLAB_OK : DPSLAB_ERR_CUDA;
}

// The dynamic shared-memory cap of a kernel is a property of the kernel, not
// of a plan: raise it to what this plan needs, never lower it (a plan created
// later with smaller grids must not break an earlier one).
void raise_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return;
    if (size_t(fa.maxDynamicSharedSizeBytes) < bytes)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

// DPSLAB_TRACE set in the environment: failing CUDA calls are reported on
// stderr with the call and its line (the return codes carry no detail)
bool trace_on() {
    static const bool on = std::getenv("DPSLAB_TRACE") != nullptr;
    return on;
}
void trace(const char* what, cudaError_t e, int line) {
    if (trace_on()) std::fprintf(stderr, "dpslab: %s failed at solve.cu:%d: %s\n", what, line, cudaGetErrorString(e));
}

#define DPS_CUDA(call)                                \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) {                      \
            trace(#call, e_, __LINE__);               \
            return cuda_err(e_);                      \
        }                                             \
    } while (0)

constexpr size_t align_up_c(size_t v) { return (v + 255) & ~size_t(255); }
size_t align_up(size_t v) { return align_up_c(v); }

template <class T>
T* carve(char*& cur, size_t count) {
    T* p = reinterpret_cast<T*>(cur);
    cur += align_up(count * sizeof(T));
    return p;
}

int floor_pow2(int v) {
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

// Column kernels by modes per block (launch-shape knob): FP64 2 or 4, mixed 4 or 8.
constexpr int kMinColBlock = 4;         // smallest mixed block; the FP64 one is half of it
using ColKernel = void (*)(KP);
ColKernel column_mixed_kernel(int cb) { return cb == 4 ? k_column_mixed<4> : k_column_mixed<8>; }
// tensor-core form: 8 W modes per block, R = ceil(N / 32) rows per lane
ColKernel column_tc_kernel(int W, int R) {
    if (R == 4) return W == 1 ? k_column_tc<1, 4> : W == 2 ? k_column_tc<2, 4> : k_column_tc<4, 4>;
    return W == 1 ? k_column_tc<1, 8> : W == 2 ? k_column_tc<2, 8> : k_column_tc<4, 8>;
}
// the persistent grid of the tensor-core form's column kernel: its blocks
// resident on all SMs at once (at most one per block of modes); 0 (one block
// per block of modes) for the other forms or when the query fails
void col_grid_update(dpslab_plan* pl) {
    pl->col_grid = 0;
    if (!pl->ztensor) return;
    int nsm = 0, per = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pl->device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per, reinterpret_cast<const void*>(column_tc_kernel(pl->col_cb / 8, pl->tc_r)), 8 * pl->col_cb,
            pl->sm_col) != cudaSuccess ||
        per < 1 || nsm < 1)
        return;
    pl->col_grid = std::min(pl->kp.n_col_blocks, per * nsm);
}
using ColBatchKernel = void (*)(ColBatch);
ColBatchKernel column_tc_batch_kernel(int W, int R) {
    if (R == 4) return W == 1 ? k_column_tc_batch<1, 4> : W == 2 ? k_column_tc_batch<2, 4> : k_column_tc_batch<4, 4>;
    return W == 1 ? k_column_tc_batch<1, 8> : W == 2 ? k_column_tc_batch<2, 8> : k_column_tc_batch<4, 8>;
}
size_t tc_smem(int nz, int W) {
    return size_t(8 * W) * size_t(tc_stride(nz)) * (sizeof(float4) + sizeof(float2)) + size_t(kTcTables) * nz * sizeof(float);
}
ColKernel column_kernel(int cb) { return cb == 2 ? k_column<2> : k_column<4>; }
// dynamic shared memory of the column kernel with cb modes per block
size_t col_smem(const dpslab_plan* pl, int cb) {
    const int nz = pl->kp.nz;
    const bool mixed = pl->kp.mixed != 0;
    if (pl->ztensor) return tc_smem(nz, cb / 8);
    const size_t rsz = mixed ? sizeof(float) : sizeof(double), csz = 2 * rsz;
    return size_t(cb) * (nz + (mixed ? ((2 - nz) & 15) : 0)) * (4 * csz + 2 * rsz);
}
using SpreadKernel = void (*)(KP);
SpreadKernel spread_mixed_kernel(int cpt) {
    return cpt == 1 ? k_spread_f32<1> : cpt == 2 ? k_spread_f32<2> : k_spread_f32<4>;
}

// Carve the plan's workspace from base (every per-solve device array: grids,
// charge arrays, buckets, cell list, partial sums); with base == nullptr it
// only measures. Returns the bytes used.
size_t bind_work(dpslab_plan* pl, char* base) {
    KP& kp = pl->kp;
    const size_t n = size_t(pl->max_n), rsz = pl->rsz;
    const size_t M = size_t(kp.ny) * kp.nxh;
    char* cur = base;
    kp.rho = carve<char>(cur, 2 * pl->G * rsz);
    kp.spec = carve<char>(cur, 2 * pl->S * 2 * rsz);
    kp.specB = carve<char>(cur, pl->S * 2 * rsz);
    kp.fields = carve<char>(cur, pl->G * 4 * rsz);
    kp.part = carve<double4_32a>(cur, n);
    kp.far = carve<double4_32a>(cur, n);
    kp.nearv = carve<double4_32a>(cur, n);
    kp.cell_of = carve<int>(cur, n);
    kp.sorted_idx = carve<int>(cur, n);
    kp.sorted = carve<double4_32a>(cur, n);
    kp.sorted_rel = carve<float4>(cur, n);
    kp.irec = carve<IRec>(cur, n);
    kp.srcs_tmp = kp.mixed ? carve<SrcF>(cur, 3 * n) : nullptr;
    kp.colp = pl->ztensor ? carve<ColP>(cur, M) : nullptr;
    kp.zcol = kp.mixed ? carve<double>(cur, 2 * size_t(kp.nz) + 1) : nullptr;
    kp.tile_count = carve<int>(cur, size_t(kp.nbuckets) + 1);
    kp.tile_start = carve<int>(cur, size_t(kp.nbuckets) + 1);
    kp.tile_fill = carve<int>(cur, size_t(kp.nbuckets) + 1);
    kp.srcs = reinterpret_cast<SrcRec*>(carve<char>(cur, pl->src_bytes));
    kp.srcsf = reinterpret_cast<SrcF*>(kp.srcs);
    kp.cell_count = carve<int>(cur, size_t(kp.ncells) + 1);
    kp.cell_start = carve<int>(cur, size_t(kp.ncells) + 1);
    kp.cell_fill = carve<int>(cur, size_t(kp.ncells) + 1);
    carve<int>(cur, size_t(kp.ncells));
    // one per column block, for the smallest block the autotuner may choose
    // (kMinColBlock / 2 modes: the FP64 kernel's smaller shape)
    kp.part_gauge_far = carve<double>(cur, (M + kMinColBlock / 2 - 1) / (kMinColBlock / 2));
    kp.part_gauge_near = carve<double>(cur, 2 * size_t(kp.n_charge_blocks));
    kp.part_u = carve<double>(cur, 2 * size_t(kp.n_charge_blocks));
    kp.part_q = carve<double>(cur, 2 * size_t(kp.n_charge_blocks));
    kp.part_wall = carve<double>(cur, 3 * size_t(kp.n_charge_blocks));
    kp.wall_phi = carve<double>(cur, n);
    kp.bd_steric = carve<double>(cur, 3 * n);
    kp.bd_prop = carve<double>(cur, 3 * n);
    kp.bd_wnew = carve<double>(cur, 3 * n);
    kp.bd_flags = carve<int>(cur, DPSLAB_BD_MAX_RETRIES);
    kp.scal = carve<double>(cur, 16);
    kp.status = carve<int>(cur, 16);
    pl->scan_part = carve<int>(cur, pl->scan_n);
    pl->d_pos = carve<double>(cur, 3 * n);
    pl->d_force = carve<double>(cur, 3 * n);
    pl->d_q = carve<double>(cur, n);
    pl->d_phi = carve<double>(cur, n);
    if (base) pl->bound = true;
    return size_t(cur - base);
}

void release(dpslab_plan* pl) {
    if (!pl) return;
    if (pl->done) cudaEventDestroy(pl->done);
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->ev_join) cudaEventDestroy(pl->ev_join);
    if (pl->side) cudaStreamDestroy(pl->side);
    for (auto& e : pl->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : pl->ev_near)
        if (e) cudaEventDestroy(e);
    if (pl->tables) cudaFree(pl->tables);
    if (pl->work) cudaFree(pl->work);
    if (pl->sig_mem) cudaFree(pl->sig_mem);
    if (pl->h_scal) cudaFreeHost(pl->h_scal);
    if (pl->h_status) cudaFreeHost(pl->h_status);
    delete pl;
}

}  // namespace

extern "C" int dpslab_derive(const dpslab_params* p, dpslab_derived* out) {
    if (!p || !out) return DPSLAB_ERR_INVALID_ARG;
    return dps::derive(*p, *out);
}

extern "C" int dpslab_table(const dpslab_params* p, int which, double* out, int n_out) {
    if (!p || !out) return DPSLAB_ERR_INVALID_ARG;
    dpslab_derived d;
    int rc = dps::derive(*p, d);
    if (rc) return rc;
    if (n_out < d.nz) return DPSLAB_ERR_INVALID_ARG;
    dps::Tables t;
    rc = dps::build_tables(*p, d, t);
    if (rc) return rc;
    const std::vector<double>* v = which == 0 ? &t.zn : which == 1 ? &t.wz : which == 2 ? &t.wg : nullptr;
    if (!v) return DPSLAB_ERR_INVALID_ARG;
    std::copy(v->begin(), v->end(), out);
    return DPSLAB_OK;
}

namespace {
enum PlanMode { kPlanFull = 0, kPlanDeferWork = 1, kPlanMeasure = 2 };
int plan_create_impl(const dpslab_params* p, int64_t max_n, int mode, dpslab_plan** out);
}

extern "C" int dpslab_plan_create(const dpslab_params* p, int64_t max_n, dpslab_plan** out) {
    return plan_create_impl(p, max_n, kPlanFull, out);
}

namespace {
int plan_create_impl(const dpslab_params* p, int64_t max_n, int mode, dpslab_plan** out) {
    const bool measure = mode == kPlanMeasure, defer_work = mode != kPlanFull;
    if (!out) return DPSLAB_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p || max_n < 1 || max_n > (int64_t(1) << 28)) return DPSLAB_ERR_INVALID_ARG;
    dpslab_plan* pl = new (std::nothrow) dpslab_plan();
    if (!pl) return DPSLAB_ERR_INVALID_ARG;
    pl->p = *p;
    pl->max_n = max_n;
    int rc = dps::derive(*p, pl->d);
    if (rc) { delete pl; return rc; }
    dps::Tables t;
    rc = dps::build_tables(*p, pl->d, t);
    if (rc) { delete pl; return rc; }
    if (!measure) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) { delete pl; return DPSLAB_ERR_NO_DEVICE; }
        cudaGetDevice(&pl->device);
    }

    const dpslab_derived& d = pl->d;
    const int nx = d.nx, ny = d.ny, nz = d.nz, nxh = nx / 2 + 1;
    pl->nxh = nxh;
    pl->G = size_t(nz) * ny * nx;
    pl->S = size_t(nz) * ny * nxh;
    KP& kp = pl->kp;
    kp.Lx = p->Lx; kp.Ly = p->Ly; kp.H = p->H; kp.eps = p->eps; kp.gw = p->gw;
    auto wall = [&](double ew, double& G, double& c, double& dd, double& tau, double& rtau, int& metal) {
        metal = std::isinf(ew) ? 1 : 0;
        if (metal) { G = 1.0; c = 1.0; dd = 0.0; tau = 0.0; rtau = 2.0; return; }
        const double r = ew / p->eps;
        G = (r - 1.0) / (r + 1.0); c = r / (1.0 + r); dd = 1.0 / (1.0 + r); tau = 2.0 / (1.0 + r); rtau = 2.0 * r / (1.0 + r);
    };
    wall(p->eps_b, kp.Gb, kp.cb, kp.db, kp.tb, kp.rtb, kp.metal_b);
    wall(p->eps_t, kp.Gt, kp.ct, kp.dt, kp.tt, kp.rtt, kp.metal_t);
    kp.nx = nx; kp.ny = ny; kp.nz = nz; kp.nxh = nxh;
    kp.hx = d.hx; kp.hy = d.hy; kp.HE = d.HE; kp.gt = d.gt; kp.xi = d.xi; kp.r_cut = d.r_cut;
    kp.a = d.a; kp.b = d.b; kp.Hbar = d.Hbar; kp.kmax = d.kmax;
    kp.s1norm = std::pow(2.0 * 3.14159265358979323846 * d.gt * d.gt, -0.5);
    kp.sigma2 = std::isinf(d.xi) ? 0.0 : (0.5 / d.xi) * (0.5 / d.xi);
    kp.inv_nxny = 1.0 / (double(nx) * double(ny));
    kp.f.kxs = float(2.0 * 3.14159265358979323846 / p->Lx);
    kp.f.kys = float(2.0 * 3.14159265358979323846 / p->Ly);
    kp.f.H = float(p->H); kp.f.HE = float(d.HE); kp.f.Hbar = float(d.Hbar); kp.f.sz = float(2.0 / d.Hbar);
    kp.f.scale = float(-(0.5 * d.Hbar) * (0.5 * d.Hbar) / p->eps);
    kp.f.Gb = float(kp.Gb); kp.f.Gt = float(kp.Gt); kp.f.cb = float(kp.cb); kp.f.db = float(kp.db);
    kp.f.ct = float(kp.ct); kp.f.dt = float(kp.dt); kp.f.tb = float(kp.tb); kp.f.tt = float(kp.tt);
    kp.f.rtb = float(kp.rtb); kp.f.rtt = float(kp.rtt); kp.f.sigma2 = float(kp.sigma2);
    kp.f.hx = float(d.hx); kp.f.hy = float(d.hy); kp.f.ig2 = float(1.0 / (2.0 * d.gt * d.gt));
    kp.f.s1norm = float(kp.s1norm);
    kp.f.a = float(d.a);
    kp.near_on = d.r_cut > 0.0 && std::isfinite(d.xi);
    kp.na1 = 2.0 * p->gw;
    kp.pa1 = std::sqrt(2.0) * p->gw;
    kp.na2 = kp.near_on ? std::sqrt(kp.na1 * kp.na1 + 1.0 / (d.xi * d.xi)) : 0.0;
    kp.pa2 = kp.near_on ? std::sqrt(kp.pa1 * kp.pa1 + 1.0 / (d.xi * d.xi)) : 0.0;
    kp.near_quad = 0;
    if (kp.near_on) {
        // 4-point Gauss-Legendre on [1/a2, 1/a1] when r_cut (1/a1 - 1/a2) is small
        const double s1 = 1.0 / kp.na1, s2 = 1.0 / kp.na2, hw = 0.5 * (s1 - s2), mid = 0.5 * (s1 + s2);
        if ((s1 - s2) * d.r_cut < 0.05) {
            const double x[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563, 0.8611363115940526};
            const double w[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461, 0.3478548451374538};
            for (int i = 0; i < 4; ++i) {
                kp.gq_s[i] = float(mid + hw * x[i]);
                kp.gq_w[i] = float(hw * w[i]);
            }
            kp.near_quad = 1;
        }
    }
    kp.nradx = int(t.radx.size());
    kp.nrady = int(t.rady.size());
    for (int i = 0; i < kp.nradx; ++i) kp.radx[i] = t.radx[i];
    for (int i = 0; i < kp.nrady; ++i) kp.rady[i] = t.rady[i];
    if (kp.near_on) {
        kp.ncx = std::max(1, int(std::floor(p->Lx / d.r_cut)));
        kp.ncy = std::max(1, int(std::floor(p->Ly / d.r_cut)));
        kp.ncz = std::max(1, int(std::floor(p->H / d.r_cut)));
        if (double(kp.ncx) * kp.ncy * kp.ncz > double(1 << 26)) { delete pl; return DPSLAB_ERR_GRID; }
        kp.ncells = kp.ncx * kp.ncy * kp.ncz;
        kp.cwx = p->Lx / kp.ncx;
        kp.cwy = p->Ly / kp.ncy;
        kp.cwz = p->H / kp.ncz;
    } else {
        kp.ncx = kp.ncy = kp.ncz = 1;
        kp.ncells = 1;
        kp.cwx = p->Lx; kp.cwy = p->Ly; kp.cwz = p->H;
    }
    // spreading tiles
    kp.ntx = (nx + kTile - 1) / kTile;
    kp.nty = (ny + kTile - 1) / kTile;
    kp.ntiles = kp.ntx * kp.nty;
    {
        // a source can reach the block's tile from r tiles away; one tile more
        // when the last tile is narrower than kTile points
        const int rx = int(std::ceil(d.HE / (kTile * d.hx))) + (nx % kTile ? 1 : 0);
        const int ry = int(std::ceil(d.HE / (kTile * d.hy))) + (ny % kTile ? 1 : 0);
        kp.tile_r = std::max(rx, ry);
        if (kp.tile_r > 3) { delete pl; return DPSLAB_ERR_GRID; }
    }
    const int M = ny * nxh;
    const bool mixed = p->precision == DPSLAB_MIXED || p->precision == DPSLAB_MIXED_SIMT;
    // z transforms on the tensor cores: Nz <= 256, and rows of a spectrum
    // plane (2 ny (nx/2+1) floats) a multiple of 16 bytes for the bulk copies
    pl->ztensor = p->precision == DPSLAB_MIXED && nz <= kZMaxNz && (M % 2) == 0 && !t.zimg_fwd.empty();
    kp.slab = mixed ? kSlabM : 16;
    kp.nslabs = (nz + kp.slab - 1) / kp.slab;
    kp.nbuckets = kp.ntiles * kp.nslabs;
    kp.supx = d.support_x;
    kp.supy = d.support_y;
    kp.mixed = mixed ? 1 : 0;
    kp.zspin = kZSpinLimit;
    int col_block = mixed ? kColBlockM : kColBlock;
    if (pl->ztensor) {
        // the tensor-core form's column kernel: the most modes per block whose
        // shared memory lets two blocks share an SM
        pl->tc_r = nz <= 128 ? 4 : 8;
        col_block = 8;
        for (int W = 4; W >= 1; W /= 2)
            if (2 * (tc_smem(nz, W) + 1024) <= 228 * 1024) { col_block = 8 * W; break; }
    }
    kp.n_col_blocks = (M + col_block - 1) / col_block;
    const size_t rsz = mixed ? sizeof(float) : sizeof(double);   // grid element size
    kp.n_charge_blocks = int((max_n + kChargeThreads - 1) / kChargeThreads);

    // tables (one allocation)
    {
        const size_t N = nz;
        size_t bytes = 0;
        const size_t vec = align_up(N * sizeof(double));
        bytes += 2 * vec + 4 * align_up(N * N * sizeof(double)) + 12 * vec;
        bytes += align_up(nx * sizeof(double2)) + align_up(ny * sizeof(double2));
        // float copies: cft, tie, tio (together <= 2 N^2) and 18 vectors
        bytes += 3 * align_up(N * N * sizeof(float)) + 18 * align_up(N * sizeof(float));
        if (pl->ztensor) bytes += 2 * align_up(t.zimg_fwd.size() * sizeof(unsigned short));   // bf16 images
        bytes += align_up(nx * sizeof(float2)) + align_up(ny * sizeof(float2));
        if (mixed) bytes += align_up(size_t(M) * sizeof(double4_32a));   // per-mode correction factors
        bytes += align_up(N);                                              // node masks
        if (pl->ztensor)                                                   // rho_o's pair transform
            bytes += align_up(kMaxOPairs * sizeof(int)) + align_up(size_t(kMaxOPairs) * N * sizeof(float));
        pl->device_bytes += int64_t(bytes);   // table bytes, taken up again below
    }
    if (!measure) {
        const size_t bytes = size_t(pl->device_bytes);
        pl->device_bytes = 0;
        cudaError_t e = cudaMalloc(&pl->tables, bytes);
        if (e != cudaSuccess) { release(pl); return DPSLAB_ERR_CUDA; }
        pl->device_bytes += int64_t(bytes);
        char* cur = static_cast<char*>(pl->tables);
        auto up = [&](const std::vector<double>& v, const double*& dst) {
            double* dp = carve<double>(cur, v.size());
            cudaMemcpy(dp, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
            dst = dp;
        };
        up(t.zn, kp.zn); up(t.wz, kp.wz);
        up(t.cft, kp.cft); up(t.tie, kp.tie); up(t.tio, kp.tio);
        up(t.j2l, kp.j2l); up(t.j2d, kp.j2d); up(t.j2u, kp.j2u);
        up(t.u1, kp.u1); up(t.u2, kp.u2); up(t.v1, kp.v1); up(t.v2, kp.v2);
        up(t.t0, kp.t0); up(t.tH, kp.tH); up(t.wg, kp.wg); up(t.wgH, kp.wgH);
        double2* tx = carve<double2>(cur, nx);
        double2* ty = carve<double2>(cur, ny);
        cudaMemcpy(tx, t.twx.data(), nx * sizeof(double2), cudaMemcpyHostToDevice);
        cudaMemcpy(ty, t.twy.data(), ny * sizeof(double2), cudaMemcpyHostToDevice);
        kp.twx = tx;
        kp.twy = ty;
        auto upf = [&](const std::vector<double>& v, const float*& dst) {
            std::vector<float> f(v.begin(), v.end());
            float* dp = carve<float>(cur, f.size());
            cudaMemcpy(dp, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
            dst = dp;
        };
        upf(t.zn, kp.zn32);
        kp.node_mask = nullptr;
        kp.o_pairs = 0;
        kp.o_pair = nullptr;
        kp.o_fwd = nullptr;
        if (pl->ztensor) {
            // bit 0, the nodes rho_o can reach: a charge of C_over lies in
            // (0, 2 H_E] or [H - 2 H_E, H), its support within H_E of it; bit
            // 1, the nodes the interpolation reads: within H_E of a charge in
            // (0, H) (a relative margin of 1e-6 keeps every node the
            // spreading's and the interpolation's test admits)
            const double he = d.HE * (1.0 + 1e-6), H = p->H;
            const size_t N = size_t(nz);
            std::vector<unsigned char> on(N);
            for (size_t j = 0; j < N; ++j) {
                const double z = t.zn[j];
                const bool o = (z >= -he && z <= 3.0 * he) || (z >= H - 3.0 * he && z <= H + he);
                const bool f = z >= -he && z <= H + he;
                on[j] = (o ? 1 : 0) | (f ? 2 : 0);
            }
            unsigned char* dp = carve<unsigned char>(cur, N);
            cudaMemcpy(dp, on.data(), N, cudaMemcpyHostToDevice);
            kp.node_mask = dp;
            // rho_o's coefficients from its node pairs (a, m - a), a <= m - a,
            // either node reachable: the forward transform of the extrema
            // grid (DCT-I form), fhat_n = (2/m) w_n sum_j w_j v_j cos(pi n j/m),
            // w = 1/2 at the ends, by the symmetry cos(pi n (m - a)/m) =
            // (-1)^n cos(pi n a/m); with more than kMaxOPairs pairs (or N not
            // a multiple of 8) the z transform keeps rho_o
            const int m = int(N) - 1;
            std::vector<int> pairs;
            for (int a = 0; 2 * a <= m; ++a)
                if ((on[a] | on[m - a]) & 1) pairs.push_back(a);
            int* pp = carve<int>(cur, kMaxOPairs);
            float* fw = carve<float>(cur, size_t(kMaxOPairs) * N);
            kp.o_pairs = 0;
            if (!pairs.empty() && int(pairs.size()) <= kMaxOPairs && m > 0 && N % 8 == 0) {
                std::vector<float> tab(pairs.size() * N);
                for (size_t q = 0; q < pairs.size(); ++q) {
                    const int a = pairs[q];
                    const double wa = (a == 0 || a == m) ? 0.5 : 1.0;
                    for (int n = 0; n < int(N); ++n) {
                        const double wn = (n == 0 || n == m) ? 0.5 : 1.0;
                        const double ang = 3.14159265358979323846 * double((size_t(n) * a) % (2 * size_t(m))) / m;
                        tab[q * N + n] = float(2.0 / m * wa * wn * std::cos(ang));
                    }
                }
                cudaMemcpy(pp, pairs.data(), pairs.size() * sizeof(int), cudaMemcpyHostToDevice);
                cudaMemcpy(fw, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice);
                kp.o_pairs = int(pairs.size());
            }
            kp.o_pair = pp;
            kp.o_fwd = fw;
        }
        {
            std::vector<double> hinv(t.zn.size(), 0.0);
            for (size_t j = 1; j < hinv.size(); ++j) hinv[j] = 0.5 / double(j);
            upf(hinv, kp.hinv32);
        }
        if (pl->ztensor) {
            auto upimg = [&](const std::vector<unsigned short>& v, const unsigned short*& dst) {
                unsigned short* dp = carve<unsigned short>(cur, v.size());
                cudaMemcpy(dp, v.data(), v.size() * sizeof(unsigned short), cudaMemcpyHostToDevice);
                dst = dp;
            };
            upimg(t.zimg_fwd, kp.zimg_fwd);
            upimg(t.zimg_inv, kp.zimg_inv);
        }
        {
            std::vector<double> lo(t.zn.size()), wzh(t.wz.size());
            for (size_t j = 0; j < t.zn.size(); ++j) lo[j] = t.zn[j] - double(float(t.zn[j]));
            for (size_t j = 0; j < t.wz.size(); ++j) wzh[j] = t.wz[j] * d.hx * d.hy;
            upf(lo, kp.znlo32);
            upf(wzh, kp.wzh32);
        }
        upf(t.cft, kp.cft32); upf(t.tie, kp.tie32); upf(t.tio, kp.tio32);
        upf(t.j2l, kp.j2l32); upf(t.j2d, kp.j2d32); upf(t.j2u, kp.j2u32);
        upf(t.u1, kp.u132); upf(t.u2, kp.u232); upf(t.v1, kp.v132); upf(t.v2, kp.v232);
        upf(t.t0, kp.t032); upf(t.tH, kp.tH32); upf(t.wg, kp.wg32);
        {
            // (J^T v)_m = a(m+1) v_{m+1} + b(m-1) v_{m-1}: row n of J has
            // 1/(2n) at n-1 and -1/(2n) at n+1 for n >= 2, 1 at 0 and -1/2 at
            // 2 for n = 1, and nothing for n = 0; columns stop at N-1
            const int nn = int(t.t0.size());
            auto jt = [&](const std::vector<double>& v) {
                std::vector<double> o(nn, 0.0);
                for (int m = 0; m < nn; ++m) {
                    if (m + 1 < nn) o[m] += (m + 1 == 1 ? 1.0 : 0.5 / (m + 1)) * v[m + 1];
                    if (m - 1 >= 1) o[m] += (m - 1 == 1 ? -0.5 : -0.5 / (m - 1)) * v[m - 1];
                }
                return o;
            };
            const std::vector<double> j0 = jt(t.t0), jj0 = jt(j0), jH = jt(t.tH), jjH = jt(jH);
            upf(j0, kp.jt0_32); upf(jj0, kp.jjt0_32); upf(jH, kp.jtH_32); upf(jjH, kp.jjtH_32);
        }
        auto upc = [&](const std::vector<dps::Complex>& v, const float2*& dst) {
            std::vector<float2> f(v.size());
            for (size_t i = 0; i < v.size(); ++i) f[i] = make_float2(float(v[i].re), float(v[i].im));
            float2* dp = carve<float2>(cur, f.size());
            cudaMemcpy(dp, f.data(), f.size() * sizeof(float2), cudaMemcpyHostToDevice);
            dst = dp;
        };
        upc(t.twx, kp.twx32);
        upc(t.twy, kp.twy32);
        if (mixed) {
            // per mode, in extended precision: k, e^{-kH}, 1/den and
            // -(1 - Gt e^{-2kH})/den, den = 1 - Gb Gt e^{-2kH}; both
            // differences from 1 are formed as (1 - G) - G expm1(-2kH), which
            // does not cancel as k -> 0 with G -> 1 (metal walls, small eps_w)
            std::vector<double4_32a> mt(static_cast<size_t>(M));
            const long double Gb = kp.Gb, Gt = kp.Gt, H = p->H;
            for (int col = 0; col < M; ++col) {
                const int iy = col / kp.nxh, ix = col - iy * kp.nxh;
                const int my = iy < (ny + 1) / 2 ? iy : iy - ny;
                const long double kx = 2.0L * 3.141592653589793238462643383279503L * ix / p->Lx;
                const long double ky = 2.0L * 3.141592653589793238462643383279503L * my / p->Ly;
                const long double k = sqrtl(kx * kx + ky * ky);
                if (k == 0.0L) {
                    mt[col] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
                    continue;
                }
                const long double e = expl(-k * H), em = expm1l(-2.0L * k * H);
                const long double den = (1.0L - Gb * Gt) - Gb * Gt * em;
                const long double ct = (1.0L - Gt) - Gt * em;
                mt[col] = make_double4_32a(double(k), double(e), double(1.0L / den), double(-ct / den));
            }
            double4_32a* dp = carve<double4_32a>(cur, mt.size());
            cudaMemcpy(dp, mt.data(), mt.size() * sizeof(double4_32a), cudaMemcpyHostToDevice);
            kp.mtab = dp;
            k_mode_flags<<<(M + 255) / 256, 256>>>(kp, dp);
            if (cudaStreamSynchronize(0) != cudaSuccess) { release(pl); return DPSLAB_ERR_CUDA; }
        }
        if (cudaGetLastError() != cudaSuccess) { release(pl); return DPSLAB_ERR_CUDA; }
    }
    // work space: sizes of the worst-case arrays, then one allocation (or,
    // for plans of a batch, a workspace shared with the other plans of its
    // stream, bound later)
    {
        const size_t n = size_t(max_n);
        // source records, worst case. FP64: every source in every slab.
        // Mixed: a source is stored once per (tile, slab) block it touches.
        size_t src_bytes = size_t(3 * n) * size_t(kp.nslabs) * sizeof(SrcRec);
        if (mixed) {
            const int spc = p->H <= 4.0 * d.HE ? 3 : 2;     // charge and its images
            auto axis = [](int sup, int nn) {
                const int tl = (sup - 1 + kTile - 1) / kTile + 1 + (nn % kTile ? 1 : 0);
                return std::min(tl, (nn + kTile - 1) / kTile);
            };
            int maxnodes = 1;                                 // nodes in any window of width 2 H_E
            for (int j0 = 0, j1 = 0; j0 < nz; ++j0) {
                while (j1 + 1 < nz && t.zn[j0] - t.zn[j1 + 1] <= 2.0 * d.HE * (1.0 + 1e-12)) ++j1;
                maxnodes = std::max(maxnodes, j1 - j0 + 1);
            }
            const int sl = std::min(kp.nslabs, (maxnodes - 1) / kSlabM + 2);
            const size_t recs = n * size_t(spc) * size_t(axis(d.support_x, nx)) * size_t(axis(d.support_y, ny)) * size_t(sl);
            src_bytes = recs * sizeof(SrcF);
            kp.src_cap = recs;
        }
        pl->src_bytes = src_bytes;
        pl->rsz = rsz;
        pl->scan_n = 2 * ((std::max<size_t>(kp.nbuckets, kp.ncells) + kScanChunk - 1) / kScanChunk + 1);
        pl->work_bytes = bind_work(pl, nullptr);
        if (measure) {
            pl->device_bytes += int64_t(pl->work_bytes);
            *out = pl;
            return DPSLAB_OK;
        }
        if (!defer_work) {
            cudaError_t e = cudaMalloc(&pl->work, pl->work_bytes);
            if (e != cudaSuccess) { release(pl); return DPSLAB_ERR_CUDA; }
            pl->device_bytes += int64_t(pl->work_bytes);
            bind_work(pl, static_cast<char*>(pl->work));
            // rho_o at the nodes it cannot reach is never written: zero once
            // (nothing reads it; this keeps the grid clean for inspection)
            if (cudaMemset(kp.rho, 0, 2 * pl->G * rsz) != cudaSuccess) { release(pl); return DPSLAB_ERR_CUDA; }
        }
    }
    if (cudaMallocHost(&pl->h_scal, 16 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&pl->h_status, 16 * sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        release(pl);
        return DPSLAB_ERR_CUDA;
    }

    // launch shapes and shared memory
    pl->px_fwd = std::max(1, std::min(8, 3072 / nx));
    pl->tk_fwd = std::max(1, std::min(16, floor_pow2(std::max(1, 3072 / ny))));
    pl->tk_inv = std::max(1, std::min(8, floor_pow2(std::max(1, 1024 / ny))));
    pl->px_inv = std::max(1, std::min(8, 1536 / nx));
    const size_t csz = 2 * rsz;                               // complex element size
    pl->sm_fftx_fwd = (size_t(nx) + 2 * size_t(pl->px_fwd) * nx) * csz;
    pl->sm_ffty_fwd = (size_t(ny) + 2 * size_t(pl->tk_fwd) * ny) * csz;
    pl->sm_ffty_inv = (size_t(ny) + 6 * size_t(pl->tk_inv) * ny) * csz;
    pl->sm_fftx_inv = (size_t(nx) + 4 * size_t(pl->px_inv) * nx) * csz;
    // power-of-two sizes: register radix-16 kernels, one slot of 16 values
    // per thread, one padded buffer (n + n/16 elements) per sequence
    {
        const size_t cap = 200 * 1024;
        auto pow2 = [](int v) { return v >= 32 && v <= kMaxFft && (v & (v - 1)) == 0; };
        // largest block each kernel can launch with (its register count)
        auto maxthr = [](const void* f) {
            cudaFuncAttributes fa{};
            return cudaFuncGetAttributes(&fa, f) == cudaSuccess ? fa.maxThreadsPerBlock : 0;
        };
        auto lg = [](int v) { int l = 0; while ((1 << l) < v) ++l; return l; };
        auto p2k = [&](int which, int n) {
            return (const void*)(mixed ? fft_p2<float>(which, lg(n)) : fft_p2<double>(which, lg(n)));
        };
        const int mxf = pow2(nx) ? maxthr(p2k(0, nx)) : 0, mxi = pow2(nx) ? maxthr(p2k(3, nx)) : 0;
        const int myf = pow2(ny) ? maxthr(p2k(1, ny)) : 0, myi = pow2(ny) ? maxthr(p2k(2, ny)) : 0;
        if (pow2(nx)) {
            const int n16 = nx / 16;
            // the inverse pairs its two sequences per row across lanes (8 elements more each)
            const size_t seq = size_t(nx + n16) * csz, seq_inv = size_t(nx + n16 + 8) * csz;
            const int P = std::max(1, std::min(256, mxf) / n16), Pi = std::max(1, std::min(128, mxi) / (2 * n16));
            const size_t fwd = P * seq, inv = 2 * Pi * seq_inv;   // the twiddle table is read from global memory
            if (fwd <= cap && inv <= cap && P * n16 <= mxf && 2 * Pi * n16 <= mxi) {
                pl->p2x = 1;
                pl->lognx = lg(nx);
                pl->px_fwd = P;
                pl->px_inv = Pi;
                pl->sm_fftx_fwd = fwd;
                pl->sm_fftx_inv = inv;
                pl->thr_x_fwd = P * n16;
                pl->thr_x_inv = 2 * Pi * n16;
            }
        }
        if (pow2(ny)) {
            const int n16 = ny / 16;
            const size_t seq = size_t(ny + n16) * csz, tw = size_t(ny) * csz;
            int T = std::max(1, std::min(8, myf / n16)), Ti = std::max(1, std::min(8, myi / n16));
            while (T > 1 && tw + T * seq > cap) T /= 2;
            while (Ti > 1 && tw + Ti * seq > cap) Ti /= 2;
            if (tw + T * seq <= cap && tw + Ti * seq <= cap && T * n16 <= myf && Ti * n16 <= myi) {
                pl->p2y = 1;
                pl->logny = lg(ny);
                pl->tk_fwd = T;
                pl->tk_inv = Ti;
                pl->sm_ffty_fwd = tw + T * seq;
                pl->sm_ffty_inv = tw + Ti * seq;
                pl->thr_y_fwd = T * n16;
                pl->thr_y_inv = Ti * n16;
            }
        }
    }
    pl->col_cb = col_block;
    pl->spread_cpt = mixed ? kSpreadCptM : 1;
    pl->sm_col = col_smem(pl, col_block);
    pl->sm_interp = size_t(pl->interp_warps) * (2 * kMaxSupport + kMaxNz) * rsz;
    pl->sm_spread = (2 * size_t(kp.slab) * kTile * kTile +
                     size_t(kSpreadBatch) * (((kp.supx + 31) & ~31) + ((kp.supy + 31) & ~31) + kp.slab)) * rsz;
    const size_t smax = 227 * 1024;
    if (pl->sm_fftx_fwd > smax || pl->sm_ffty_fwd > smax || pl->sm_ffty_inv > smax ||
        pl->sm_fftx_inv > smax || pl->sm_col > smax || pl->sm_spread > smax) {
        release(pl);
        return DPSLAB_ERR_GRID;
    }
    if (mixed) {
        if (pl->p2x) {
            raise_smem(reinterpret_cast<const void*>(fft_p2<float>(0, pl->lognx)), size_t(pl->sm_fftx_fwd));
            raise_smem(reinterpret_cast<const void*>(fft_p2<float>(3, pl->lognx)), size_t(pl->sm_fftx_inv));
        }
        if (pl->p2y) {
            raise_smem(reinterpret_cast<const void*>(fft_p2<float>(1, pl->logny)), size_t(pl->sm_ffty_fwd));
            raise_smem(reinterpret_cast<const void*>(fft_p2<float>(2, pl->logny)), size_t(pl->sm_ffty_inv));
        }
        raise_smem(reinterpret_cast<const void*>(k_fftx_fwd<float>), size_t(pl->sm_fftx_fwd));
        raise_smem(reinterpret_cast<const void*>(k_ffty_fwd<float>), size_t(pl->sm_ffty_fwd));
        raise_smem(reinterpret_cast<const void*>(k_ffty_inv<float>), size_t(pl->sm_ffty_inv));
        raise_smem(reinterpret_cast<const void*>(k_fftx_inv<float>), size_t(pl->sm_fftx_inv));
        if (pl->ztensor) {
            raise_smem(reinterpret_cast<const void*>(k_zgemm_fwd), size_t(kZSmem));
            raise_smem(reinterpret_cast<const void*>(k_zgemm_inv), size_t(kZSmem));
            int nsm = 0;
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pl->device);
            const int ntiles = 2 * int((2 * size_t(M) + kZN - 1) / kZN);   // both planes
            pl->zgrid = std::max(1, std::min(ntiles, nsm));
        }
        if (pl->ztensor) {
            for (int W = 1; W <= 4; W *= 2)
                if (tc_smem(nz, W) <= 227 * 1024)
                    raise_smem(reinterpret_cast<const void*>(column_tc_kernel(W, pl->tc_r)), tc_smem(nz, W));
        } else {
            for (int cb = kMinColBlock; cb <= kColBlockM; cb *= 2)
                raise_smem(reinterpret_cast<const void*>(column_mixed_kernel(cb)), col_smem(pl, cb));
        }
        col_grid_update(pl);
        raise_smem(reinterpret_cast<const void*>(k_interp_f32),
                   size_t(kMaxInterpWarps) * (2 * kMaxSupport + kMaxNz) * sizeof(float));
    } else {
        if (pl->p2x) {
            raise_smem(reinterpret_cast<const void*>(fft_p2<double>(0, pl->lognx)), size_t(pl->sm_fftx_fwd));
            raise_smem(reinterpret_cast<const void*>(fft_p2<double>(3, pl->lognx)), size_t(pl->sm_fftx_inv));
        }
        if (pl->p2y) {
            raise_smem(reinterpret_cast<const void*>(fft_p2<double>(1, pl->logny)), size_t(pl->sm_ffty_fwd));
            raise_smem(reinterpret_cast<const void*>(fft_p2<double>(2, pl->logny)), size_t(pl->sm_ffty_inv));
        }
        raise_smem(reinterpret_cast<const void*>(k_fftx_fwd<double>), size_t(pl->sm_fftx_fwd));
        raise_smem(reinterpret_cast<const void*>(k_ffty_fwd<double>), size_t(pl->sm_ffty_fwd));
        raise_smem(reinterpret_cast<const void*>(k_ffty_inv<double>), size_t(pl->sm_ffty_inv));
        raise_smem(reinterpret_cast<const void*>(k_fftx_inv<double>), size_t(pl->sm_fftx_inv));
        for (int cb = kMinColBlock / 2; cb <= kColBlock; cb *= 2)
            raise_smem(reinterpret_cast<const void*>(column_kernel(cb)), col_smem(pl, cb));
        raise_smem(reinterpret_cast<const void*>(k_interp<double>), size_t(pl->sm_interp));
        raise_smem(reinterpret_cast<const void*>(k_spread_tiled<double>), size_t(pl->sm_spread));
    }
    if (cudaGetLastError() != cudaSuccess) { release(pl); return DPSLAB_ERR_CUDA; }
    *out = pl;
    return DPSLAB_OK;
}
}  // namespace

extern "C" int dpslab_plan_derived(const dpslab_plan* plan, dpslab_derived* out) {
    if (!plan || !out) return DPSLAB_ERR_INVALID_ARG;
    *out = plan->d;
    return DPSLAB_OK;
}

extern "C" int64_t dpslab_plan_device_bytes(const dpslab_plan* plan) { return plan ? plan->device_bytes : 0; }

extern "C" int dpslab_plan_create_unbound(const dpslab_params* p, int64_t max_n, dpslab_plan** out) {
    return plan_create_impl(p, max_n, kPlanDeferWork, out);
}

extern "C" int64_t dpslab_plan_work_bytes(const dpslab_plan* plan) { return plan ? int64_t(plan->work_bytes) : 0; }

extern "C" int dpslab_plan_bind_work(dpslab_plan* plan, void* work, int64_t bytes) {
    if (!plan || plan->work || plan->in_flight) return DPSLAB_ERR_INVALID_ARG;   // owned workspace, or busy
    if (!work) {
        plan->bound = false;
        return DPSLAB_OK;
    }
    if (reinterpret_cast<uintptr_t>(work) % 256 != 0 || bytes < int64_t(plan->work_bytes)) return DPSLAB_ERR_INVALID_ARG;
    bind_work(plan, static_cast<char*>(work));
    return DPSLAB_OK;
}

namespace {
// forward and inverse xy transforms of the plan's grids, launched as a solve
// launches them (used by the wall-charge set-up)
template <class R>
int xy_transforms(dpslab_plan* pl, const KP& kp, cudaStream_t st, bool inverse) {
    const int npairs = kp.nz * kp.ny;
    if (!inverse) {
        const dim3 gy((kp.nxh + pl->tk_fwd - 1) / pl->tk_fwd, 2 * kp.nz);
        const int gx = (npairs + pl->px_fwd - 1) / pl->px_fwd;
        if (pl->p2x) fft_p2<R>(0, pl->lognx)<<<gx, pl->thr_x_fwd, pl->sm_fftx_fwd, st>>>(kp, pl->px_fwd, pl->lognx);
        else k_fftx_fwd<R><<<gx, 256, pl->sm_fftx_fwd, st>>>(kp, pl->px_fwd);
        if (pl->p2y) fft_p2<R>(1, pl->logny)<<<gy, pl->thr_y_fwd, pl->sm_ffty_fwd, st>>>(kp, pl->tk_fwd, pl->logny);
        else k_ffty_fwd<R><<<gy, 256, pl->sm_ffty_fwd, st>>>(kp, pl->tk_fwd);
    } else {
        const dim3 gy((kp.nxh + pl->tk_inv - 1) / pl->tk_inv, kp.nz);
        const int gx = (npairs + pl->px_inv - 1) / pl->px_inv;
        if (pl->p2y) fft_p2<R>(2, pl->logny)<<<gy, pl->thr_y_inv, pl->sm_ffty_inv, st>>>(kp, pl->tk_inv, pl->logny);
        else k_ffty_inv<R><<<gy, 256, pl->sm_ffty_inv, st>>>(kp, pl->tk_inv);
        if (pl->p2x) fft_p2<R>(3, pl->lognx)<<<gx, pl->thr_x_inv, pl->sm_fftx_inv, st>>>(kp, pl->px_inv, pl->lognx);
        else k_fftx_inv<R><<<gx, 256, pl->sm_fftx_inv, st>>>(kp, pl->px_inv);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        trace("xy_transforms", e, __LINE__);
        return DPSLAB_ERR_CUDA;
    }
    return DPSLAB_OK;
}

// transforms of the wall charges, the potential grid of their correction and
// its own energy term, on the plan's workspace (Eq. (mm2), (mm4), (Ufinal))
template <class R>
int wall_setup(dpslab_plan* pl, const double* planes, cudaStream_t st) {
    KP kp = pl->kp;
    kp.node_mask = nullptr;   // the set-up transforms every plane
    const int M = kp.ny * kp.nxh;
    const size_t G = size_t(kp.nz) * kp.ny * kp.nx, P2 = 2 * size_t(kp.ny) * kp.nx;
    char* base = static_cast<char*>(pl->sig_mem);
    double2* hat = reinterpret_cast<double2*>(base);
    R* grid = reinterpret_cast<R*>(base + align_up(2 * size_t(M) * sizeof(double2)));
    double* tmp = reinterpret_cast<double*>(reinterpret_cast<char*>(grid) + align_up(G * sizeof(R)));
    double* self = tmp + P2;
    DPS_CUDA(cudaMemcpyAsync(tmp, planes, P2 * sizeof(double), cudaMemcpyHostToDevice, st));
    DPS_CUDA(cudaMemsetAsync(kp.rho, 0, 2 * G * sizeof(R), st));
    k_wall_fill<R><<<unsigned((P2 + 255) / 256), 256, 0, st>>>(kp, tmp);
    if (int rc = xy_transforms<R>(pl, kp, st, false)) return rc;
    k_wall_hat<R><<<(2 * M + 255) / 256, 256, 0, st>>>(kp, hat);
    k_wall_nodes<R><<<unsigned((size_t(kp.nz) * M + 255) / 256), 256, 0, st>>>(kp, hat);
    if (int rc = xy_transforms<R>(pl, kp, st, true)) return rc;
    k_wall_grid<R><<<unsigned((G + 255) / 256), 256, 0, st>>>(kp, grid);
    k_wall_self<<<1, 1024, 0, st>>>(kp, hat, self);
    DPS_CUDA(cudaGetLastError());
    double h[3];
    DPS_CUDA(cudaMemcpyAsync(&h[0], &hat[0].x, sizeof(double), cudaMemcpyDeviceToHost, st));
    DPS_CUDA(cudaMemcpyAsync(&h[1], &hat[M].x, sizeof(double), cudaMemcpyDeviceToHost, st));
    DPS_CUDA(cudaMemcpyAsync(&h[2], self, sizeof(double), cudaMemcpyDeviceToHost, st));
    DPS_CUDA(cudaStreamSynchronize(st));
    pl->kp.sig_hat = hat;
    pl->kp.sig_grid = grid;
    pl->kp.sig_Qb = kp.hx * kp.hy * h[0];
    pl->kp.sig_Qt = kp.hx * kp.hy * h[1];
    pl->kp.sig_self = h[2];
    pl->kp.sigma_on = 1;
    return DPSLAB_OK;
}
}  // namespace

extern "C" int dpslab_plan_set_wall_charge(dpslab_plan* plan, const double* sigma_b, const double* sigma_t,
                                           void* stream) {
    if (!plan || plan->in_flight || !plan->bound) return DPSLAB_ERR_INVALID_ARG;
    DPS_CUDA(cudaSetDevice(plan->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    KP& kp = plan->kp;
    if (!sigma_b && !sigma_t) {
        kp.sigma_on = 0;
        if (plan->sig_mem) {
            DPS_CUDA(cudaStreamSynchronize(st));
            cudaFree(plan->sig_mem);
            plan->sig_mem = nullptr;
            plan->device_bytes -= int64_t(plan->sig_bytes);
            plan->sig_bytes = 0;
        }
        return DPSLAB_OK;
    }
    if ((sigma_b && kp.metal_b) || (sigma_t && kp.metal_t)) return DPSLAB_ERR_UNSUPPORTED;
    const size_t P1 = size_t(kp.ny) * kp.nx, G = size_t(kp.nz) * P1, M = size_t(kp.ny) * kp.nxh;
    std::vector<double> planes(2 * P1, 0.0);
    for (size_t i = 0; i < P1; ++i) {
        const double b = sigma_b ? sigma_b[i] : 0.0, t = sigma_t ? sigma_t[i] : 0.0;
        if (!std::isfinite(b) || !std::isfinite(t)) return DPSLAB_ERR_INVALID_ARG;
        planes[i] = b;
        planes[P1 + i] = t;
    }
    if (!plan->sig_mem) {
        const size_t bytes = align_up(2 * M * sizeof(double2)) + align_up(G * plan->rsz) + align_up(2 * P1 * sizeof(double)) +
                             align_up(sizeof(double));
        if (cudaMalloc(&plan->sig_mem, bytes) != cudaSuccess) {
            plan->sig_mem = nullptr;
            return DPSLAB_ERR_CUDA;
        }
        plan->sig_bytes = bytes;
        plan->device_bytes += int64_t(bytes);
    }
    kp.sigma_on = 0;
    return kp.mixed ? wall_setup<float>(plan, planes.data(), st) : wall_setup<double>(plan, planes.data(), st);
}

// ---------------------------------------------------------------------------
// Brownian dynamics, Sec. 7.1: Eq. (leimkuhler), (steric), (lj)
// ---------------------------------------------------------------------------
namespace {
// Which part of a solve enqueue() issues: all of it, or (for batches, whose
// column stage is one launch over several systems) the part before the
// column stage or the part after it.
enum SolvePart { kSolveAll = 0, kSolveFront = 1, kSolveBack = 2 };
int enqueue(dpslab_plan* pl, int64_t n64, const double* pos, const double* q, double* phi, double* force,
            cudaStream_t st, SolvePart part = kSolveAll);
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;   // Philox4x32 multipliers
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;   // key increments

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011)
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        const uint32_t hi0 = __umulhi(kPhiloxM0, c[0]), lo0 = kPhiloxM0 * c[0];
        const uint32_t hi1 = __umulhi(kPhiloxM1, c[2]), lo1 = kPhiloxM1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// W_i at (step, retry): the generator's four words as uniforms (w + 1/2) 2^-32,
// two Box-Muller pairs, the first three numbers
__device__ __forceinline__ double3 bd_normals(uint32_t i, uint64_t step, uint32_t retry, uint64_t seed) {
    uint32_t c[4] = {i, uint32_t(step), uint32_t(step >> 32), retry};
    philox4x32_10(c, uint32_t(seed), uint32_t(seed >> 32));
    const double s = 2.3283064365386962890625e-10;   // 2^-32
    const double u0 = (double(c[0]) + 0.5) * s, u1 = (double(c[1]) + 0.5) * s;
    const double u2 = (double(c[2]) + 0.5) * s, u3 = (double(c[3]) + 0.5) * s;
    const double r1 = sqrt(-2.0 * log(u0)), r2 = sqrt(-2.0 * log(u2));
    return make_double3(r1 * cos(kTwoPi * u1), r1 * sin(kTwoPi * u1), r2 * cos(kTwoPi * u3));
}

struct BdConst {
    double dt, mu, amp, a2, U0, r_m, rs2, max_disp;
    int p, R;
    uint64_t seed, step;
};

// Eq. (steric): F_LJ(max(r, r_m)) for r <= 2^(1/p) 2a (caller checks the range)
__device__ __forceinline__ double bd_steric_mag(double r, const BdConst& b) {
    const double rr = fmax(r, b.r_m);
    double s = 1.0;
    const double t = b.a2 / rr;
    for (int k = 0; k < b.p; ++k) s *= t;
    return 4.0 * b.U0 * b.p / rr * (2.0 * s * s - s);
}

__global__ void k_bd_init(uint64_t seed, int n, double* W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double3 w = bd_normals(uint32_t(i), 0, 0, seed);
    W[3 * i] = w.x;
    W[3 * i + 1] = w.y;
    W[3 * i + 2] = w.z;
}

// steric forces at z^n on the solve's cell list (cells are at least r_cut >=
// 2^(1/p) 2a wide), plus each ion's own wall images
__global__ void k_bd_steric(KP kp, BdConst b) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= kp.n) return;
    const double4_32a t = kp.sorted[s];
    const int cx = min(kp.ncx - 1, max(0, int(t.x / kp.cwx)));
    const int cy = min(kp.ncy - 1, max(0, int(t.y / kp.cwy)));
    const int cz = min(kp.ncz - 1, max(0, int(t.z / kp.cwz)));
    const int nxc = kp.ncx >= 3 ? 3 : kp.ncx, nyc = kp.ncy >= 3 ? 3 : kp.ncy;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int zc = max(0, cz - 1); zc <= min(kp.ncz - 1, cz + 1); ++zc) {
        for (int oy = 0; oy < nyc; ++oy) {
            const int yc = kp.ncy >= 3 ? wrap_index(cy - 1 + oy, kp.ncy) : oy;
            for (int ox = 0; ox < nxc; ++ox) {
                const int xc = kp.ncx >= 3 ? wrap_index(cx - 1 + ox, kp.ncx) : ox;
                const int cell = cell_index(kp, xc, yc, zc);
                for (int u = kp.cell_start[cell]; u < kp.cell_start[cell + 1]; ++u) {
                    if (u == s) continue;
                    const double4_32a o = kp.sorted[u];
                    const double dx = min_image(t.x - o.x, kp.Lx), dy = min_image(t.y - o.y, kp.Ly), dz = t.z - o.z;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 <= b.rs2) {
                        const double r = sqrt(r2), f = bd_steric_mag(r, b) / r;
                        fx = fma(f, dx, fx);
                        fy = fma(f, dy, fy);
                        fz = fma(f, dz, fz);
                    }
                }
            }
        }
    }
    const double db = 2.0 * t.z, dt = 2.0 * (kp.H - t.z);
    if (db * db <= b.rs2) fz += bd_steric_mag(db, b);
    if (dt * dt <= b.rs2) fz -= bd_steric_mag(dt, b);
    const int k = kp.sorted_idx[s];
    kp.bd_steric[3 * k] = fx;
    kp.bd_steric[3 * k + 1] = fy;
    kp.bd_steric[3 * k + 2] = fz;
}

__device__ __forceinline__ bool bd_skip(const KP& kp, int r) {
    if (*kp.status & (kStatusOutOfSlab | kStatusNonFinite)) return true;   // the solve refused z^n
    for (int rr = 0; rr < r; ++rr)
        if (kp.bd_flags[rr] == 0) return true;                             // an earlier proposal was accepted
    return false;
}

// proposal r of Eq. (leimkuhler) from the sanitised z^n; flags it if an ion leaves 0 < z < H
__global__ void k_bd_propose(KP kp, BdConst b, const double* F, const double* W, int r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kp.n || bd_skip(kp, r)) return;
    const double4_32a p = kp.part[i];
    const double3 wn = bd_normals(uint32_t(i), b.step + 1, uint32_t(r), b.seed);
    const double* fs = kp.bd_steric + 3 * i;
    double dx = b.mu * (F[3 * i] + fs[0]) * b.dt + b.amp * (W[3 * i] + wn.x);
    double dy = b.mu * (F[3 * i + 1] + fs[1]) * b.dt + b.amp * (W[3 * i + 1] + wn.y);
    double dz = b.mu * (F[3 * i + 2] + fs[2]) * b.dt + b.amp * (W[3 * i + 2] + wn.z);
    if (b.max_disp > 0.0) {
        const double nrm = sqrt(dx * dx + dy * dy + dz * dz);
        if (nrm > b.max_disp) {
            const double sc = b.max_disp / nrm;
            dx *= sc;
            dy *= sc;
            dz *= sc;
        }
    }
    const double z = p.z + dz;
    kp.bd_prop[3 * i] = np_mod(p.x + dx, kp.Lx);
    kp.bd_prop[3 * i + 1] = np_mod(p.y + dy, kp.Ly);
    kp.bd_prop[3 * i + 2] = z;
    kp.bd_wnew[3 * i] = wn.x;
    kp.bd_wnew[3 * i + 1] = wn.y;
    kp.bd_wnew[3 * i + 2] = wn.z;
    if (!(z > 0.0 && z < kp.H)) atomicOr(&kp.bd_flags[r], 1);
}

// accept proposal r if no ion left the slab (and none before was accepted)
__global__ void k_bd_commit(KP kp, BdConst b, double* pos, double* W, int r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (bd_skip(kp, r)) return;
    if (kp.bd_flags[r] != 0) {
        if (r == b.R - 1 && i == 0) {
            atomicOr(kp.status, kStatusRejected);
            kp.scal[9] = double(b.R);
        }
        return;
    }
    if (i == 0) kp.scal[9] = double(r);
    if (i >= kp.n) return;
    for (int c = 0; c < 3; ++c) {
        pos[3 * i + c] = kp.bd_prop[3 * i + c];
        W[3 * i + c] = kp.bd_wnew[3 * i + c];
    }
}
}  // namespace

extern "C" int dpslab_bd_init_noise(uint64_t seed, int64_t n, double* W, void* stream) {
    if (!W || n < 1 || n > (int64_t(1) << 31) - 1) return DPSLAB_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_bd_init<<<unsigned((n + 255) / 256), 256, 0, st>>>(seed, int(n), W);
    DPS_CUDA(cudaGetLastError());
    return DPSLAB_OK;
}

extern "C" int dpslab_bd_step_enqueue(dpslab_plan* plan, const dpslab_bd_params* bp, int64_t n, double* pos,
                                      const double* q, double* W, uint64_t step, double* force, void* stream) {
    if (!plan || !bp || !pos || !q || !W || n < 1 || plan->in_flight || !plan->bound) return DPSLAB_ERR_INVALID_ARG;
    if (n > plan->max_n) return DPSLAB_ERR_CAPACITY;
    const KP& kp0 = plan->kp;
    const double rs = std::pow(2.0, 1.0 / std::max(1, bp->p)) * 2.0 * bp->a;
    if (!(bp->dt > 0.0) || !(bp->mu > 0.0) || !(bp->kT >= 0.0) || !(bp->a > 0.0) || !(bp->U0 >= 0.0) ||
        !(bp->r_m > 0.0) || bp->p < 1 || bp->max_retries < 1 || bp->max_retries > DPSLAB_BD_MAX_RETRIES ||
        !(bp->max_disp >= 0.0) || !kp0.near_on || rs > kp0.r_cut)
        return DPSLAB_ERR_INVALID_ARG;
    DPS_CUDA(cudaSetDevice(plan->device));
    if (!plan->done) DPS_CUDA(cudaEventCreateWithFlags(&plan->done, cudaEventDisableTiming));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* F = force ? force : plan->d_force;
    const int prof = plan->profiling;
    plan->profiling = 0;
    int rc = enqueue(plan, n, pos, q, nullptr, F, st);
    plan->profiling = prof;
    if (rc) return rc;
    KP kp = plan->kp;
    kp.n = int(n);
    kp.pos = pos;
    kp.q = q;
    BdConst b;
    b.dt = bp->dt;
    b.mu = bp->mu;
    b.amp = std::sqrt(bp->kT * bp->mu * bp->dt / 2.0);
    b.a2 = 2.0 * bp->a;
    b.U0 = bp->U0;
    b.r_m = bp->r_m;
    b.rs2 = rs * rs;
    b.max_disp = bp->max_disp;
    b.p = bp->p;
    b.R = bp->max_retries;
    b.seed = bp->seed;
    b.step = step;
    const int nb = int((n + 255) / 256);
    DPS_CUDA(cudaMemsetAsync(kp.bd_flags, 0, DPSLAB_BD_MAX_RETRIES * sizeof(int), st));
    k_bd_steric<<<nb, 256, 0, st>>>(kp, b);
    for (int r = 0; r < b.R; ++r) {
        k_bd_propose<<<nb, 256, 0, st>>>(kp, b, F, W, r);
        k_bd_commit<<<nb, 256, 0, st>>>(kp, b, pos, W, r);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        trace("bd kernels", e, __LINE__);
        return DPSLAB_ERR_CUDA;
    }
    plan->launches += 1 + 2 * b.R;
    DPS_CUDA(cudaMemcpyAsync(plan->h_scal, kp.scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
    DPS_CUDA(cudaMemcpyAsync(plan->h_status, kp.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DPS_CUDA(cudaEventRecord(plan->done, st));
    plan->last_n = n;
    plan->in_flight = true;
    return DPSLAB_OK;
}

extern "C" int dpslab_bd_last_retries(const dpslab_plan* plan) {
    return plan ? int(plan->h_scal[9]) : 0;
}

extern "C" int dpslab_plan_footprint(const dpslab_params* p, int64_t max_n, int64_t* bytes) {
    if (!bytes) return DPSLAB_ERR_INVALID_ARG;
    *bytes = 0;
    dpslab_plan* pl = nullptr;
    const int rc = plan_create_impl(p, max_n, kPlanMeasure, &pl);
    if (rc) return rc;
    *bytes = pl->device_bytes;
    delete pl;        // measure mode holds no device or pinned memory
    return DPSLAB_OK;
}

extern "C" int dpslab_plan_destroy(dpslab_plan* plan) {
    if (!plan) return DPSLAB_OK;
    cudaSetDevice(plan->device);
    release(plan);
    return DPSLAB_OK;
}

extern "C" int dpslab_last_launch_count(const dpslab_plan* plan) { return plan ? plan->launches : 0; }

extern "C" int dpslab_plan_set_wait_limit(dpslab_plan* plan, int64_t polls) {
    if (!plan || polls < 0 || plan->in_flight) return DPSLAB_ERR_INVALID_ARG;
    plan->kp.zspin = polls;
    return DPSLAB_OK;
}

// stage events (created on first use)
int make_stage_events(dpslab_plan* plan) {
    if (!plan->ev[0]) {
        for (auto& e : plan->ev) DPS_CUDA(cudaEventCreate(&e));
        for (auto& e : plan->ev_near) DPS_CUDA(cudaEventCreate(&e));
    }
    return DPSLAB_OK;
}

extern "C" int dpslab_profile(dpslab_plan* plan, int on) {
    if (!plan || on < 0 || on > 2) return DPSLAB_ERR_INVALID_ARG;
    DPS_CUDA(cudaSetDevice(plan->device));
    if (on) {
        const int rc = make_stage_events(plan);
        if (rc) return rc;
    }
    plan->profiling = on;
    return DPSLAB_OK;
}

extern "C" int dpslab_stage_times(const dpslab_plan* plan, double* ms, int n) {
    if (!plan || !ms || n < DPSLAB_NSTAGES) return DPSLAB_ERR_INVALID_ARG;
    for (int i = 0; i < DPSLAB_NSTAGES; ++i) ms[i] = plan->stage_ms[i];
    return DPSLAB_OK;
}

// ---------------------------------------------------------------------------
// launch-shape autotuning (the xy transforms' sequences per block)
// ---------------------------------------------------------------------------
namespace {
int finish(dpslab_plan* pl, cudaStream_t st, double* U);
// x forward, y forward, y inverse, x inverse transforms; interpolation;
// column kernel; spreading (DPSLAB_NKNOBS)
constexpr int kKnobs = DPSLAB_NKNOBS;
constexpr int kKnobStage[kKnobs] = {2, 3, 7, 8, 9, 5, 1};

int* shape_knob(dpslab_plan* pl, int which) {
    switch (which) {
        case 0: return &pl->px_fwd;
        case 1: return &pl->tk_fwd;
        case 2: return &pl->tk_inv;
        case 3: return &pl->px_inv;
        case 4: return &pl->interp_warps;
        case 5: return &pl->col_cb;
        default: return &pl->spread_cpt;
    }
}

// knobs 4-6: warps per block of the interpolation (1, 2, 4, 8), modes per
// block of the column kernel (mixed 4 or 8, FP64 2 or 4), x columns per
// thread of the mixed spreading (1 or 2; FP64 1)
bool apply_kernel_knob(dpslab_plan* pl, int which, int v) {
    const bool mixed = pl->kp.mixed != 0;
    const size_t rsz = mixed ? sizeof(float) : sizeof(double);
    if (which == 4) {
        if (v != 1 && v != 2 && v != 4 && v != kMaxInterpWarps) return false;
        const size_t sm = size_t(v) * (2 * kMaxSupport + kMaxNz) * rsz;
        if (!mixed) {
            raise_smem(reinterpret_cast<const void*>(k_interp<double>), sm);
            raise_smem(reinterpret_cast<const void*>(k_wall_cross<double>), sm);
        } else {
            raise_smem(reinterpret_cast<const void*>(k_wall_cross<float>), sm);
        }
        pl->interp_warps = v;
        pl->sm_interp = sm;
        return true;
    }
    if (which == 5) {
        if (pl->ztensor) {
            if (v != 8 && v != 16 && v != 32) return false;
        } else {
            const int lo = mixed ? kMinColBlock : kMinColBlock / 2, hi = mixed ? kColBlockM : kColBlock;
            if (v != lo && v != hi) return false;
        }
        const size_t sm = col_smem(pl, v);
        if (sm > 227 * 1024) return false;
        const int M = pl->kp.ny * pl->kp.nxh;
        pl->col_cb = v;
        pl->sm_col = sm;
        pl->kp.n_col_blocks = (M + v - 1) / v;
        col_grid_update(pl);
        return true;
    }
    if (v != 1 && !(mixed && (v == 2 || v == 4))) return false;
    pl->spread_cpt = v;
    return true;
}

// set knob `which` to v sequences per block, with its block size and shared
// memory; false (nothing changed) outside the kernel's thread and shared-memory limits
template <class R>
bool apply_shape_t(dpslab_plan* pl, int which, int v) {
    if (v < 1 || v > 64) return false;
    const size_t csz = 2 * sizeof(R), smax = 227 * 1024;
    const int nx = pl->kp.nx, ny = pl->kp.ny;
    auto maxthr = [](const void* f) {
        cudaFuncAttributes fa{};
        return cudaFuncGetAttributes(&fa, f) == cudaSuccess ? fa.maxThreadsPerBlock : 0;
    };
    const bool xk = which == 0 || which == 3;
    const int n = xk ? nx : ny;
    const bool p2 = xk ? pl->p2x : pl->p2y;
    size_t sm;
    int thr = 256;
    const void* f;
    if (p2) {
        const int n16 = n / 16;
        // x transforms read the global twiddle table, y transforms a shared copy
        const size_t seq = size_t(n + n16 + (which == 3 ? 8 : 0)) * csz,
                     tw = which == 1 || which == 2 ? size_t(n) * csz : 0;
        const int seqs = which == 3 ? 2 * v : v;         // the x inverse transforms two sequences per row
        thr = seqs * n16;
        sm = tw + seqs * seq;
        f = (const void*)fft_p2<R>(which, which == 0 || which == 3 ? pl->lognx : pl->logny);
        if (thr > maxthr(f)) return false;
    } else {
        const int mul = which == 0 || which == 1 ? 2 : which == 2 ? 6 : 4;
        sm = (size_t(n) + size_t(mul) * v * n) * csz;
        f = which == 0 ? (const void*)k_fftx_fwd<R> : which == 1 ? (const void*)k_ffty_fwd<R>
          : which == 2 ? (const void*)k_ffty_inv<R> : (const void*)k_fftx_inv<R>;
    }
    if (sm > smax) return false;
    raise_smem(f, sm);
    *shape_knob(pl, which) = v;
    switch (which) {
        case 0: pl->sm_fftx_fwd = sm; pl->thr_x_fwd = thr; break;
        case 1: pl->sm_ffty_fwd = sm; pl->thr_y_fwd = thr; break;
        case 2: pl->sm_ffty_inv = sm; pl->thr_y_inv = thr; break;
        default: pl->sm_fftx_inv = sm; pl->thr_x_inv = thr; break;
    }
    return true;
}

bool apply_shape(dpslab_plan* pl, int which, int v) {
    if (which >= 4) return apply_kernel_knob(pl, which, v);
    return pl->kp.mixed ? apply_shape_t<float>(pl, which, v) : apply_shape_t<double>(pl, which, v);
}
}  // namespace

extern "C" int dpslab_plan_tuning(const dpslab_plan* plan, int* knobs, int n) {
    if (!plan || !knobs || n < 4) return DPSLAB_ERR_INVALID_ARG;
    for (int i = 0; i < std::min(n, kKnobs); ++i) knobs[i] = *shape_knob(const_cast<dpslab_plan*>(plan), i);
    return DPSLAB_OK;
}

extern "C" int dpslab_plan_set_tuning(dpslab_plan* plan, const int* knobs, int n) {
    if (!plan || !knobs || n < 4 || plan->in_flight) return DPSLAB_ERR_INVALID_ARG;
    DPS_CUDA(cudaSetDevice(plan->device));
    int old[kKnobs];
    dpslab_plan_tuning(plan, old, kKnobs);
    for (int i = 0; i < std::min(n, kKnobs); ++i) {
        if (!apply_shape(plan, i, knobs[i])) {
            for (int j = 0; j < i; ++j) apply_shape(plan, j, old[j]);
            return DPSLAB_ERR_INVALID_ARG;
        }
    }
    return DPSLAB_OK;
}

extern "C" int dpslab_plan_autotune(dpslab_plan* plan, int64_t n, const double* pos, const double* q, int reps,
                                    void* stream) {
    if (!plan || !pos || !q || n < 1 || reps < 1 || plan->in_flight || !plan->bound) return DPSLAB_ERR_INVALID_ARG;
    if (n > plan->max_n) return DPSLAB_ERR_CAPACITY;
    DPS_CUDA(cudaSetDevice(plan->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (const int erc = make_stage_events(plan)) return erc;
    const int prof = plan->profiling;
    plan->profiling = 2;   // stage times with nothing running beside them
    // median stage time of `reps` solves after one warm-up
    auto time_stage = [&](int stage, double& out) -> int {
        std::vector<double> t;
        for (int i = 0; i <= reps; ++i) {
            int rc = enqueue(plan, n, pos, q, nullptr, nullptr, st);
            if (!rc) rc = finish(plan, st, nullptr);
            if (rc && rc != DPSLAB_ERR_NOT_NEUTRAL) return rc;
            if (i) t.push_back(plan->stage_ms[stage]);
        }
        std::sort(t.begin(), t.end());
        out = t[t.size() / 2];
        return DPSLAB_OK;
    };
    int rc = DPSLAB_OK;
    for (int which = 0; which < kKnobs && !rc; ++which) {
        const int cur = *shape_knob(plan, which);
        int best = cur;
        double tbest = 0.0;
        rc = time_stage(kKnobStage[which], tbest);
        for (int v = 1; v <= 32 && !rc; v *= 2) {
            if (v == cur || !apply_shape(plan, which, v)) continue;
            double t = 0.0;
            rc = time_stage(kKnobStage[which], t);
            if (!rc && t < 0.98 * tbest) {
                tbest = t;
                best = v;
            }
        }
        apply_shape(plan, which, best);
    }
    plan->profiling = prof;
    plan->last_n = n;
    return rc;
}

extern "C" const char* dpslab_stage_name(int stage) {
    static const char* names[DPSLAB_NSTAGES] = {"prepare", "spread", "fft_x_fwd", "fft_y_fwd", "z_fwd", "bvp",
                                                "z_inv", "fft_y_inv", "fft_x_inv", "interp", "near", "finish"};
    return (stage >= 0 && stage < DPSLAB_NSTAGES) ? names[stage] : "";
}

extern "C" const char* dpslab_strerror(int code) {
    switch (code) {
        case DPSLAB_OK: return "ok";
        case DPSLAB_ERR_INVALID_ARG: return "invalid argument";
        case DPSLAB_ERR_NOT_NEUTRAL: return "charges are not neutral";
        case DPSLAB_ERR_OUT_OF_SLAB: return "a charge lies outside 0 < z < H or is not finite";
        case DPSLAB_ERR_CUTOFF_TOO_LARGE: return "near-field cutoff not below half the period";
        case DPSLAB_ERR_SPLIT_CONSTRAINT: return "splitting constraint violated (strict mode)";
        case DPSLAB_ERR_CAPACITY: return "more charges than the plan was created for";
        case DPSLAB_ERR_CUDA: return "CUDA runtime error";
        case DPSLAB_ERR_NO_DEVICE: return "no CUDA device";
        case DPSLAB_ERR_GRID: return "grid too small for the Gaussian support or unsupported size";
        case DPSLAB_ERR_UNSUPPORTED: return "unsupported option";
        case DPSLAB_PENDING: return "the solve has not finished yet";
        case DPSLAB_ERR_BD_REJECTED: return "every proposal of the Brownian-dynamics step left the slab";
        case DPSLAB_ERR_TIMEOUT: return "a bounded wait on the tensor-core pipeline gave up";
        default: return "unknown error";
    }
}

namespace {

int enqueue(dpslab_plan* pl, int64_t n64, const double* pos, const double* q, double* phi, double* force,
            cudaStream_t st, SolvePart part) {
    KP kp = pl->kp;
    const int n = int(n64);
    kp.n = n;
    kp.pos = pos;
    kp.q = q;
    kp.out_phi = phi;
    kp.out_force = force;
    const int nb = (n + kChargeThreads - 1) / kChargeThreads;
    kp.n_charge_blocks = nb;
    int launches = part == kSolveBack ? pl->launches : 0;
    const bool prof = pl->profiling != 0;
    const bool front = part != kSolveBack, back = part != kSolveFront, column = part == kSolveAll;
    auto mark = [&](int i) {
        if (prof) cudaEventRecord(pl->ev[i], st);
    };
#define LAUNCH(...)                                  \
    do {                                             \
        __VA_ARGS__;                                 \
        ++launches;                                  \
        const cudaError_t le_ = cudaGetLastError();  \
        if (le_ != cudaSuccess) {                    \
            trace(#__VA_ARGS__, le_, __LINE__);      \
            return DPSLAB_ERR_CUDA;                  \
        }                                            \
    } while (0)
    // exclusive scan count[0..m) -> start[0..m] (m >= 1)
    auto scan = [&](const int* count, int* start, int m) -> int {
        const int nbs = (m + kScanChunk - 1) / kScanChunk;
        int* sums = pl->scan_part;
        int* offs = pl->scan_part + nbs + 1;
        LAUNCH(k_scan_sums<<<nbs, kScanBlock, 0, st>>>(count, m, sums));
        LAUNCH(k_scan<<<1, 1024, 0, st>>>(sums, offs, nbs));
        LAUNCH(k_scan_apply<<<nbs, kScanBlock, 0, st>>>(count, start, m, offs));
        return 0;
    };
#define SCAN(c, s_, m)                          \
    do {                                        \
        if (const int e_ = scan(c, s_, m)) return e_; \
    } while (0)

    const bool fork = kp.near_on && pl->profiling != 2;
    if (front) {
    DPS_CUDA(cudaMemsetAsync(kp.status, 0, sizeof(int), st));
    DPS_CUDA(cudaMemsetAsync(kp.tile_count, 0, (size_t(kp.nbuckets) + 1) * sizeof(int), st));
    DPS_CUDA(cudaMemsetAsync(kp.tile_fill, 0, (size_t(kp.nbuckets) + 1) * sizeof(int), st));
    if (kp.near_on) {
        DPS_CUDA(cudaMemsetAsync(kp.cell_count, 0, (size_t(kp.ncells) + 1) * sizeof(int), st));
        DPS_CUDA(cudaMemsetAsync(kp.cell_fill, 0, (size_t(kp.ncells) + 1) * sizeof(int), st));
    }
    mark(0);
    LAUNCH(k_prepare<<<nb, kChargeThreads, 0, st>>>(kp));
    if (kp.near_on) {   // cell list: the near field's pairs and the interpolation's order
        SCAN(kp.cell_count, kp.cell_start, kp.ncells);
        LAUNCH(k_scatter_cells<<<nb, kChargeThreads, 0, st>>>(kp));
    }
    mark(1);
    // The near field needs only the cell list (and writes only nearv): it
    // runs on the plan's second stream while the far field runs here, and
    // this stream waits for it before the assembly. Profiling mode 1 keeps
    // that and times the near field by its own events on the second stream;
    // mode 2 runs it in line, so that the stage times add up to the solve.
    pl->near_timed = fork && prof;
    if (fork) {
        DPS_CUDA(cudaEventRecord(pl->ev_fork, st));
        DPS_CUDA(cudaStreamWaitEvent(pl->side, pl->ev_fork, 0));
        if (prof) DPS_CUDA(cudaEventRecord(pl->ev_near[0], pl->side));
        if (kp.mixed) LAUNCH(k_near_f32<<<(n + 127) / 128, 128, 0, pl->side>>>(kp));
        else LAUNCH(k_near<double><<<(n + 127) / 128, 128, 0, pl->side>>>(kp));
        if (prof) DPS_CUDA(cudaEventRecord(pl->ev_near[1], pl->side));
        // the near potential at the origin (the gauge) needs only the
        // charges: beside the far field too (with wall charges it also
        // needs their interpolation, so it stays on the solve's stream)
        if (!kp.sigma_on) LAUNCH(k_origin<<<nb, kChargeThreads, 0, pl->side>>>(kp));
        DPS_CUDA(cudaEventRecord(pl->ev_join, pl->side));
    }
    const dim3 gs(kp.ntiles, kp.nslabs);
    if (kp.mixed) {
        LAUNCH(k_sources_f<<<nb, kChargeThreads, 0, st>>>(kp));
        SCAN(kp.tile_count, kp.tile_start, kp.nbuckets);
        LAUNCH(k_scatter_sources_f<<<nb, kChargeThreads, 0, st>>>(kp));
        LAUNCH(spread_mixed_kernel(pl->spread_cpt)<<<gs, kTile * kTile / pl->spread_cpt, 0, st>>>(kp));
    } else {
        LAUNCH(k_count_sources<<<nb, kChargeThreads, 0, st>>>(kp));
        SCAN(kp.tile_count, kp.tile_start, kp.nbuckets);
        LAUNCH(k_scatter_sources<<<nb, kChargeThreads, 0, st>>>(kp));
        LAUNCH(k_spread_tiled<double><<<gs, kTile * kTile, pl->sm_spread, st>>>(kp));
    }
    mark(2);
    }
    const int npairs = kp.nz * kp.ny;
    const dim3 gy_fwd((kp.nxh + pl->tk_fwd - 1) / pl->tk_fwd, 2 * kp.nz);
    const dim3 gy_inv((kp.nxh + pl->tk_inv - 1) / pl->tk_inv, kp.nz);
    const int gx_fwd = (npairs + pl->px_fwd - 1) / pl->px_fwd;
    const int gx_inv = (kp.nz * kp.ny + pl->px_inv - 1) / pl->px_inv;
    const int iw = pl->interp_warps, gi = (n + iw - 1) / iw;
    if (kp.mixed) {
        if (front) {
        if (pl->p2x) LAUNCH(fft_p2<float>(0, pl->lognx)<<<gx_fwd, pl->thr_x_fwd, pl->sm_fftx_fwd, st>>>(kp, pl->px_fwd, pl->lognx));
        else LAUNCH(k_fftx_fwd<float><<<gx_fwd, 256, pl->sm_fftx_fwd, st>>>(kp, pl->px_fwd));
        mark(3);
        if (pl->p2y) LAUNCH(fft_p2<float>(1, pl->logny)<<<gy_fwd, pl->thr_y_fwd, pl->sm_ffty_fwd, st>>>(kp, pl->tk_fwd, pl->logny));
        else LAUNCH(k_ffty_fwd<float><<<gy_fwd, 256, pl->sm_ffty_fwd, st>>>(kp, pl->tk_fwd));
        mark(4);
        LAUNCH(k_column_zero<<<1, kZeroThreads, 0, st>>>(kp));
        if (pl->ztensor) LAUNCH(k_zgemm_fwd<<<pl->zgrid, kZThreads, kZSmem, st>>>(kp));
        if (pl->ztensor && kp.o_pairs > 0)
            LAUNCH(k_o_coeffs<<<(kp.ny * kp.nxh + kOcCols - 1) / kOcCols, 256, 0, st>>>(kp));
        mark(5);
        }
        if (column) {
        if (pl->ztensor)
            LAUNCH(column_tc_kernel(pl->col_cb / 8, pl->tc_r)<<<pl->col_grid > 0 ? pl->col_grid : kp.n_col_blocks, 8 * pl->col_cb, pl->sm_col, st>>>(kp));
        else
            LAUNCH(column_mixed_kernel(pl->col_cb)<<<kp.n_col_blocks, 32 * pl->col_cb, pl->sm_col, st>>>(kp));
        }
        if (back) {
        mark(6);
        if (pl->ztensor) LAUNCH(k_zgemm_inv<<<pl->zgrid, kZThreads, kZSmem, st>>>(kp));
        mark(7);
        if (pl->p2y) LAUNCH(fft_p2<float>(2, pl->logny)<<<gy_inv, pl->thr_y_inv, pl->sm_ffty_inv, st>>>(kp, pl->tk_inv, pl->logny));
        else LAUNCH(k_ffty_inv<float><<<gy_inv, 256, pl->sm_ffty_inv, st>>>(kp, pl->tk_inv));
        mark(8);
        if (pl->p2x) LAUNCH(fft_p2<float>(3, pl->lognx)<<<gx_inv, pl->thr_x_inv, pl->sm_fftx_inv, st>>>(kp, pl->px_inv, pl->lognx));
        else LAUNCH(k_fftx_inv<float><<<gx_inv, 256, pl->sm_fftx_inv, st>>>(kp, pl->px_inv));
        mark(9);
        LAUNCH(k_interp_f32<<<gi, 32 * iw, pl->sm_interp, st>>>(kp));
        if (kp.sigma_on) LAUNCH(k_wall_cross<float><<<gi, 32 * iw, pl->sm_interp, st>>>(kp));
        }
    } else {
        if (front) {
        if (pl->p2x) LAUNCH(fft_p2<double>(0, pl->lognx)<<<gx_fwd, pl->thr_x_fwd, pl->sm_fftx_fwd, st>>>(kp, pl->px_fwd, pl->lognx));
        else LAUNCH(k_fftx_fwd<double><<<gx_fwd, 256, pl->sm_fftx_fwd, st>>>(kp, pl->px_fwd));
        mark(3);
        if (pl->p2y) LAUNCH(fft_p2<double>(1, pl->logny)<<<gy_fwd, pl->thr_y_fwd, pl->sm_ffty_fwd, st>>>(kp, pl->tk_fwd, pl->logny));
        else LAUNCH(k_ffty_fwd<double><<<gy_fwd, 256, pl->sm_ffty_fwd, st>>>(kp, pl->tk_fwd));
        mark(4);
        mark(5);
        }
        if (column) LAUNCH(column_kernel(pl->col_cb)<<<kp.n_col_blocks, 32 * pl->col_cb, pl->sm_col, st>>>(kp));
        if (back) {
        mark(6);
        mark(7);
        if (pl->p2y) LAUNCH(fft_p2<double>(2, pl->logny)<<<gy_inv, pl->thr_y_inv, pl->sm_ffty_inv, st>>>(kp, pl->tk_inv, pl->logny));
        else LAUNCH(k_ffty_inv<double><<<gy_inv, 256, pl->sm_ffty_inv, st>>>(kp, pl->tk_inv));
        mark(8);
        if (pl->p2x) LAUNCH(fft_p2<double>(3, pl->lognx)<<<gx_inv, pl->thr_x_inv, pl->sm_fftx_inv, st>>>(kp, pl->px_inv, pl->lognx));
        else LAUNCH(k_fftx_inv<double><<<gx_inv, 256, pl->sm_fftx_inv, st>>>(kp, pl->px_inv));
        mark(9);
        LAUNCH(k_interp<double><<<gi, 32 * iw, pl->sm_interp, st>>>(kp));
        if (kp.sigma_on) LAUNCH(k_wall_cross<double><<<gi, 32 * iw, pl->sm_interp, st>>>(kp));
        }
    }
    if (!back) {
        pl->launches = launches;
        return DPSLAB_OK;
    }
    mark(10);
    if (kp.near_on && !fork) {
        if (kp.mixed) LAUNCH(k_near_f32<<<(n + 127) / 128, 128, 0, st>>>(kp));
        else LAUNCH(k_near<double><<<(n + 127) / 128, 128, 0, st>>>(kp));
    }
    if (fork) DPS_CUDA(cudaStreamWaitEvent(st, pl->ev_join, 0));
    mark(11);
    if (!fork || kp.sigma_on) LAUNCH(k_origin<<<nb, kChargeThreads, 0, st>>>(kp));
    LAUNCH(k_final_gauge<<<1, 1024, 0, st>>>(kp));
    LAUNCH(k_assemble<<<nb, kChargeThreads, 0, st>>>(kp));
    LAUNCH(k_final_energy<<<1, 1024, 0, st>>>(kp));
    mark(12);
#undef LAUNCH
#undef SCAN
    DPS_CUDA(cudaMemcpyAsync(pl->h_scal, kp.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    DPS_CUDA(cudaMemcpyAsync(pl->h_status, kp.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    pl->launches = launches;
    return DPSLAB_OK;
}

// the result of a completed solve: U and the status bits copied back
int collect(dpslab_plan* pl, double* U) {
    if (U) *U = pl->h_scal[4];
    if (*pl->h_status & kStatusCapacity) return DPSLAB_ERR_CAPACITY;
    if (*pl->h_status & kStatusTimeout) return DPSLAB_ERR_TIMEOUT;
    if (*pl->h_status & kStatusRejected) return DPSLAB_ERR_BD_REJECTED;
    if (*pl->h_status) return DPSLAB_ERR_OUT_OF_SLAB;
    double sq = pl->h_scal[5], saq = pl->h_scal[6];
    if (pl->kp.sigma_on) {   // Eq. (elecneu): charges and wall charges together
        sq += pl->kp.sig_Qb + pl->kp.sig_Qt;
        saq += std::fabs(pl->kp.sig_Qb) + std::fabs(pl->kp.sig_Qt);
    }
    if (std::fabs(sq) > 1e-12 * saq) return DPSLAB_ERR_NOT_NEUTRAL;
    return DPSLAB_OK;
}

int finish(dpslab_plan* pl, cudaStream_t st, double* U) {
    DPS_CUDA(cudaStreamSynchronize(st));
    if (pl->profiling) {
        for (int i = 0; i < DPSLAB_NSTAGES; ++i) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, pl->ev[i], pl->ev[i + 1]);
            pl->stage_ms[i] = ms;
        }
        if (pl->near_timed) {   // the near stage ran beside the far field
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, pl->ev_near[0], pl->ev_near[1]);
            pl->stage_ms[kStageNear] = ms;
        }
    }
    return collect(pl, U);
}

}  // namespace

extern "C" int dpslab_solve(dpslab_plan* plan, int64_t n, const double* pos, const double* q, double* U,
                            double* phi, double* force, void* stream) {
    if (!plan || !pos || !q || n < 1 || plan->in_flight || !plan->bound) return DPSLAB_ERR_INVALID_ARG;
    if (n > plan->max_n) return DPSLAB_ERR_CAPACITY;
    DPS_CUDA(cudaSetDevice(plan->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = enqueue(plan, n, pos, q, phi, force, st);
    if (rc) return rc;
    plan->last_n = n;
    return finish(plan, st, U);
}

extern "C" int dpslab_solve_enqueue(dpslab_plan* plan, int64_t n, const double* pos, const double* q, double* phi,
                                    double* force, void* stream) {
    if (!plan || !pos || !q || n < 1 || plan->in_flight || !plan->bound) return DPSLAB_ERR_INVALID_ARG;
    if (n > plan->max_n) return DPSLAB_ERR_CAPACITY;
    DPS_CUDA(cudaSetDevice(plan->device));
    if (!plan->done) DPS_CUDA(cudaEventCreateWithFlags(&plan->done, cudaEventDisableTiming));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int prof = plan->profiling;
    plan->profiling = 0;
    const int rc = enqueue(plan, n, pos, q, phi, force, st);
    plan->profiling = prof;
    if (rc) return rc;
    DPS_CUDA(cudaEventRecord(plan->done, st));
    plan->last_n = n;
    plan->in_flight = true;
    return DPSLAB_OK;
}

extern "C" int dpslab_solve_poll(dpslab_plan* plan, double* U) {
    if (!plan || !plan->in_flight) return DPSLAB_ERR_INVALID_ARG;
    const cudaError_t e = cudaEventQuery(plan->done);
    if (e == cudaErrorNotReady) return DPSLAB_PENDING;
    plan->in_flight = false;
    if (e != cudaSuccess) {
        trace("cudaEventQuery", e, __LINE__);
        return DPSLAB_ERR_CUDA;
    }
    return collect(plan, U);
}

extern "C" int dpslab_solve_host(dpslab_plan* plan, int64_t n, const double* pos, const double* q, double* U,
                                 double* phi, double* force, void* stream) {
    if (!plan || !pos || !q || n < 1 || plan->in_flight || !plan->bound) return DPSLAB_ERR_INVALID_ARG;
    if (n > plan->max_n) return DPSLAB_ERR_CAPACITY;
    DPS_CUDA(cudaSetDevice(plan->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DPS_CUDA(cudaMemcpyAsync(plan->d_pos, pos, size_t(n) * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    DPS_CUDA(cudaMemcpyAsync(plan->d_q, q, size_t(n) * sizeof(double), cudaMemcpyHostToDevice, st));
    int rc = enqueue(plan, n, plan->d_pos, plan->d_q, phi ? plan->d_phi : nullptr, force ? plan->d_force : nullptr, st);
    if (rc) return rc;
    if (phi) DPS_CUDA(cudaMemcpyAsync(phi, plan->d_phi, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (force) DPS_CUDA(cudaMemcpyAsync(force, plan->d_force, size_t(n) * 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    plan->last_n = n;
    return finish(plan, st, U);
}

extern "C" int dpslab_debug_fetch(dpslab_plan* plan, int which, void* host_dst, size_t bytes) {
    if (!plan || !host_dst) return DPSLAB_ERR_INVALID_ARG;
    DPS_CUDA(cudaSetDevice(plan->device));
    const KP& kp = plan->kp;
    const size_t n = size_t(plan->last_n);
    const void* src = nullptr;
    size_t want = 0;
    const size_t rsz = kp.mixed ? sizeof(float) : sizeof(double);
    size_t count = 0;   // grid elements to widen from float (mixed)
    switch (which) {
        case 0: src = kp.rho; want = 2 * plan->G * sizeof(double); count = 2 * plan->G; break;
        case 1: src = kp.fields; want = plan->G * 4 * sizeof(double); count = 4 * plan->G; break;
        case 2: src = kp.far; want = n * sizeof(double4_32a); break;
        case 3: src = kp.nearv; want = n * sizeof(double4_32a); break;
        case 4: {
            if (bytes != 4 * sizeof(double)) return DPSLAB_ERR_INVALID_ARG;
            double s[4];
            DPS_CUDA(cudaMemcpy(s, kp.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost));
            double o[4] = {s[0], s[1], s[2], s[3]};
            std::memcpy(host_dst, o, sizeof(o));
            return DPSLAB_OK;
        }
        default: return DPSLAB_ERR_INVALID_ARG;
    }
    if (bytes != want) return DPSLAB_ERR_INVALID_ARG;
    if (which == 3 && !kp.near_on) {
        std::memset(host_dst, 0, bytes);
        return DPSLAB_OK;
    }
    if (count && rsz == sizeof(float)) {
        std::vector<float> tmp(count);
        DPS_CUDA(cudaMemcpy(tmp.data(), src, count * sizeof(float), cudaMemcpyDeviceToHost));
        double* d = static_cast<double*>(host_dst);
        for (size_t i = 0; i < count; ++i) d[i] = tmp[i];
        return DPSLAB_OK;
    }
    DPS_CUDA(cudaMemcpy(host_dst, src, bytes, cudaMemcpyDeviceToHost));
    return DPSLAB_OK;
}

// ===========================================================================
// Near field without any allocation
// ===========================================================================
//
// For callers that cannot call cudaMalloc: code that runs where allocation
// is forbidden or unavailable (inside a custom allocator's callbacks, under
// a memory pool that must not grow, in an embedded or real-time loop that
// pre-reserves all device memory at start-up). The scratch space of the
// cell list lives in one file-scope device array, reserved when the module
// loads; every GPU that loads this library holds it until the process exits.
namespace {

constexpr int64_t kStaticMaxN = 65536;     // charges per call
constexpr int kStaticMaxCells = 65536;     // near-field cells per call
constexpr int kStaticMaxDevices = 64;
constexpr size_t kStaticBlocks = (kStaticMaxN + kChargeThreads - 1) / kChargeThreads;
constexpr size_t kStaticScratchBytes =
    3 * align_up_c(kStaticMaxN * 32) +                        // part, sorted, near results
    align_up_c(kStaticMaxN * 16) +                            // sorted_rel
    2 * align_up_c(kStaticMaxN * 4) +                         // cell_of, sorted_idx
    3 * align_up_c((kStaticMaxCells + 1) * 4) +               // cell count, start, fill
    align_up_c(2 * kStaticBlocks * 8) + align_up_c(64);       // neutrality partials, status
static_assert(kStaticScratchBytes < (8u << 20) + (512u << 10), "the documented size: about 8.3 MiB");

static __device__ __align__(256) unsigned char g_near_scratch[kStaticScratchBytes];

std::mutex g_near_scratch_mu;
void* g_near_scratch_ptr[kStaticMaxDevices] = {};

// Device address of g_near_scratch on the current device, looked up once per
// device (host code cannot use the symbol itself as an address).
int near_scratch_address(int device, char** out) {
    if (device < 0 || device >= kStaticMaxDevices) return DPSLAB_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_near_scratch_mu);
    if (!g_near_scratch_ptr[device]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_near_scratch) != cudaSuccess || !ptr) return DPSLAB_ERR_CUDA;
        g_near_scratch_ptr[device] = ptr;
    }
    *out = static_cast<char*>(g_near_scratch_ptr[device]);
    return DPSLAB_OK;
}

}  // namespace

extern "C" int dpslab_near_field_static(const dpslab_params* p, int64_t n, const double* pos, const double* q,
                                        double* out, void* stream) {
    if (!p || !pos || !q || !out || n < 1) return DPSLAB_ERR_INVALID_ARG;
    if (n > kStaticMaxN) return DPSLAB_ERR_CAPACITY;
    dpslab_derived d;
    int rc = dps::derive(*p, d);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!(d.r_cut > 0.0) || std::isinf(d.xi)) {        // no splitting: the near field is zero
        DPS_CUDA(cudaMemsetAsync(out, 0, size_t(n) * 4 * sizeof(double), st));
        return cuda_err(cudaStreamSynchronize(st));
    }
    KP kp{};
    kp.ncx = std::max(1, int(std::floor(p->Lx / d.r_cut)));
    kp.ncy = std::max(1, int(std::floor(p->Ly / d.r_cut)));
    kp.ncz = std::max(1, int(std::floor(p->H / d.r_cut)));
    if (double(kp.ncx) * kp.ncy * kp.ncz > double(kStaticMaxCells)) return DPSLAB_ERR_CAPACITY;
    int device = 0;
    DPS_CUDA(cudaGetDevice(&device));
    char* cur = nullptr;
    rc = near_scratch_address(device, &cur);
    if (rc) return rc;

    kp.Lx = p->Lx; kp.Ly = p->Ly; kp.H = p->H; kp.eps = p->eps; kp.gw = p->gw;
    auto gamma = [&](double ew) { return std::isinf(ew) ? 1.0 : (ew / p->eps - 1.0) / (ew / p->eps + 1.0); };
    kp.Gb = gamma(p->eps_b);
    kp.Gt = gamma(p->eps_t);
    kp.r_cut = d.r_cut;
    kp.near_on = 1;
    kp.na1 = 2.0 * p->gw;
    kp.na2 = std::sqrt(kp.na1 * kp.na1 + 1.0 / (d.xi * d.xi));
    kp.ncells = kp.ncx * kp.ncy * kp.ncz;
    kp.cwx = p->Lx / kp.ncx;
    kp.cwy = p->Ly / kp.ncy;
    kp.cwz = p->H / kp.ncz;
    kp.n = int(n);
    kp.pos = pos;
    kp.q = q;
    kp.part = carve<double4_32a>(cur, kStaticMaxN);
    kp.sorted = carve<double4_32a>(cur, kStaticMaxN);
    kp.nearv = carve<double4_32a>(cur, kStaticMaxN);
    kp.sorted_rel = carve<float4>(cur, kStaticMaxN);
    kp.cell_of = carve<int>(cur, kStaticMaxN);
    kp.sorted_idx = carve<int>(cur, kStaticMaxN);
    kp.cell_count = carve<int>(cur, size_t(kStaticMaxCells) + 1);
    kp.cell_start = carve<int>(cur, size_t(kStaticMaxCells) + 1);
    kp.cell_fill = carve<int>(cur, size_t(kStaticMaxCells) + 1);
    kp.part_q = carve<double>(cur, 2 * kStaticBlocks);
    kp.status = carve<int>(cur, 16);
    const int nb = int((n + kChargeThreads - 1) / kChargeThreads);
    kp.n_charge_blocks = nb;
    // the array keeps the previous call's contents: clear what accumulates
    DPS_CUDA(cudaMemsetAsync(kp.cell_count, 0, (size_t(kp.ncells) + 1) * sizeof(int), st));
    DPS_CUDA(cudaMemsetAsync(kp.cell_fill, 0, (size_t(kp.ncells) + 1) * sizeof(int), st));
    DPS_CUDA(cudaMemsetAsync(kp.status, 0, sizeof(int), st));
    k_prepare<<<nb, kChargeThreads, 0, st>>>(kp);
    k_scan_cells<<<1, 1024, 0, st>>>(kp);
    k_scatter_cells<<<nb, kChargeThreads, 0, st>>>(kp);
    k_near<double><<<int((n + 127) / 128), 128, 0, st>>>(kp);
    DPS_CUDA(cudaGetLastError());
    DPS_CUDA(cudaMemcpyAsync(out, kp.nearv, size_t(n) * 4 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    int status = 0;
    DPS_CUDA(cudaMemcpyAsync(&status, kp.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DPS_CUDA(cudaStreamSynchronize(st));
    return status ? DPSLAB_ERR_OUT_OF_SLAB : DPSLAB_OK;
}

// ===========================================================================
// batches of independent systems
// ===========================================================================
struct dpslab_batch {
    int device = 0;
    std::vector<dpslab_plan*> plans;
    std::vector<cudaStream_t> streams;
    std::vector<void*> work;               // one shared workspace per stream
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    // the graph is captured and launched on `head` (the caller's stream may be
    // the legacy default stream, which cannot be captured), ordered after the
    // caller's prior work (`in`) and before its later work (`out`)
    cudaStream_t head = nullptr;
    cudaEvent_t in = nullptr, out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> g_n;              // arguments the graph was captured with
    std::vector<const void*> g_ptr;
    int g_schedule = -1;
    int64_t device_bytes = 0;
    // The column stage (per-mode BVP and correction) of the systems of one
    // wave (the systems that have workspaces of their own: one per stream)
    // runs as one launch per kind of column kernel over all their k modes.
    struct ColGroup {
        int kind = 0;                      // 0 FP64, 1 mixed CUDA-core z transforms, 2 mixed tensor-core
        int tc_w = 0, tc_r = 0;            // kind 2: the column kernel's shape (8 W modes per block, R)
        int blocks = 0;
        size_t smem = 0;
        std::shared_ptr<ColBatch> arg;     // the launch's parameter: up to kBatchMaxSys systems
    };
    std::vector<std::vector<ColGroup>> waves;
    int launches = 0;                      // kernels of the last batch solve
    int schedule = DPSLAB_BATCH_STREAMS;   // DPSLAB_BATCH_STREAMS or DPSLAB_BATCH_WAVES
};

namespace {
void batch_release(dpslab_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto* pl : b->plans) release(pl);
    for (void* w : b->work)
        if (w) cudaFree(w);
    for (auto st : b->streams) cudaStreamDestroy(st);
    for (auto e : b->joins) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->head) cudaStreamDestroy(b->head);
    if (b->in) cudaEventDestroy(b->in);
    if (b->out) cudaEventDestroy(b->out);
    delete b;
}
}  // namespace

extern "C" int dpslab_batch_create(const dpslab_params* params, const int64_t* max_n, int count, int nstreams,
                                   dpslab_batch** out) {
    if (!params || !max_n || !out || count < 1 || nstreams < 1) return DPSLAB_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return DPSLAB_ERR_NO_DEVICE;
    auto* b = new (std::nothrow) dpslab_batch;
    if (!b) return DPSLAB_ERR_CUDA;
    cudaGetDevice(&b->device);
    const int S = std::min(nstreams, count);
    for (int i = 0; i < count; ++i) {
        dpslab_plan* pl = nullptr;
        const int rc = plan_create_impl(&params[i], max_n[i], kPlanDeferWork, &pl);
        if (rc) { batch_release(b); return rc; }
        b->plans.push_back(pl);
        b->device_bytes += pl->device_bytes;
    }
    b->work.assign(S, nullptr);
    for (int s = 0; s < S; ++s) {
        size_t need = 0;
        for (int i = s; i < count; i += S) need = std::max(need, b->plans[i]->work_bytes);
        if (cudaMalloc(&b->work[s], need) != cudaSuccess) { batch_release(b); return DPSLAB_ERR_CUDA; }
        b->device_bytes += int64_t(need);
        for (int i = s; i < count; i += S) bind_work(b->plans[i], static_cast<char*>(b->work[s]));
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { batch_release(b); return DPSLAB_ERR_CUDA; }
        b->streams.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) { batch_release(b); return DPSLAB_ERR_CUDA; }
        b->joins.push_back(ev);
    }
    // column groups: per wave of S systems, per kind (and shape) of column
    // kernel, one launch per kBatchMaxSys systems
    b->waves.assign((count + S - 1) / S, {});
    for (int w0 = 0; w0 < count; w0 += S) {
        std::vector<std::pair<int, std::vector<int>>> keyed;   // (kind, W, R) code, systems
        for (int i = w0; i < std::min(count, w0 + S); ++i) {
            const dpslab_plan* pl = b->plans[i];
            const int kind = !pl->kp.mixed ? 0 : (pl->ztensor ? 2 : 1);
            const int key = kind == 2 ? 200 + 10 * (pl->col_cb / 8) + pl->tc_r : 100 * kind;
            auto it = std::find_if(keyed.begin(), keyed.end(), [&](const auto& e) { return e.first == key; });
            if (it == keyed.end()) keyed.push_back({key, {i}});
            else it->second.push_back(i);
        }
        for (const auto& e : keyed) {
            const std::vector<int>& sys = e.second;
            for (size_t c0 = 0; c0 < sys.size(); c0 += kBatchMaxSys) {
                dpslab_batch::ColGroup cg;
                cg.kind = e.first / 100;
                if (cg.kind == 2) {
                    cg.tc_w = (e.first % 100) / 10;
                    cg.tc_r = e.first % 10;
                }
                cg.arg = std::make_shared<ColBatch>();
                ColBatch& a = *cg.arg;
                std::memset(static_cast<void*>(&a), 0, sizeof(ColBatch));
                a.nsys = int(std::min<size_t>(kBatchMaxSys, sys.size() - c0));
                for (int j = 0; j < a.nsys; ++j) {
                    const dpslab_plan* pl = b->plans[sys[c0 + j]];
                    std::memcpy(static_cast<void*>(&a.kp[j]), &pl->kp, sizeof(KP));
                    a.starts[j + 1] = a.starts[j] + pl->kp.n_col_blocks;
                    cg.smem = std::max(cg.smem, pl->sm_col);
                }
                cg.blocks = a.starts[a.nsys];
                if (cg.kind == 0) raise_smem(reinterpret_cast<const void*>(k_column_batch), cg.smem);
                if (cg.kind == 1) raise_smem(reinterpret_cast<const void*>(k_column_mixed_batch), cg.smem);
                if (cg.kind == 2) raise_smem(reinterpret_cast<const void*>(column_tc_batch_kernel(cg.tc_w, cg.tc_r)), cg.smem);
                b->waves[w0 / S].push_back(std::move(cg));
            }
        }
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->out, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->head, cudaStreamNonBlocking) != cudaSuccess) {
        batch_release(b);
        return DPSLAB_ERR_CUDA;
    }
    *out = b;
    return DPSLAB_OK;
}

extern "C" int dpslab_batch_solve(dpslab_batch* b, const int64_t* n, const double* const* pos, const double* const* q,
                                  double* U, double* const* phi, double* const* force, int* status, void* stream) {
    if (!b || !n || !pos || !q) return DPSLAB_ERR_INVALID_ARG;
    const int count = int(b->plans.size()), S = int(b->streams.size());
    std::vector<const void*> ptr;
    ptr.reserve(4 * size_t(count));
    for (int i = 0; i < count; ++i) {
        if (!pos[i] || !q[i] || n[i] < 1) return DPSLAB_ERR_INVALID_ARG;
        if (n[i] > b->plans[i]->max_n) return DPSLAB_ERR_CAPACITY;
        ptr.push_back(pos[i]);
        ptr.push_back(q[i]);
        ptr.push_back(phi ? phi[i] : nullptr);
        ptr.push_back(force ? force[i] : nullptr);
    }
    DPS_CUDA(cudaSetDevice(b->device));
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    cudaStream_t st = b->head;
    DPS_CUDA(cudaEventRecord(b->in, caller));
    DPS_CUDA(cudaStreamWaitEvent(st, b->in, 0));
    const bool same = b->exec && b->g_ptr == ptr && int(b->g_n.size()) == count &&
                      std::equal(b->g_n.begin(), b->g_n.end(), n) && b->g_schedule == b->schedule;
    if (!same) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        DPS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = DPSLAB_OK;
        int launches = 0;
        // the streams of systems w0 .. w0 + S - 1 wait for `st`, or `st` for them
        auto fork = [&](int w0) {
            if (!rc && cudaEventRecord(b->fork, st) != cudaSuccess) rc = DPSLAB_ERR_CUDA;
            for (int s = 0; s < S && !rc && w0 + s < count; ++s)
                if (cudaStreamWaitEvent(b->streams[s], b->fork, 0) != cudaSuccess) rc = DPSLAB_ERR_CUDA;
        };
        auto join = [&](int w0) {
            for (int s = 0; s < S && !rc && w0 + s < count; ++s)
                if (cudaEventRecord(b->joins[s], b->streams[s]) != cudaSuccess ||
                    cudaStreamWaitEvent(st, b->joins[s], 0) != cudaSuccess)
                    rc = DPSLAB_ERR_CUDA;
        };
        if (b->schedule == DPSLAB_BATCH_STREAMS) {
            // every system's whole solve on its stream; the streams run freely
            fork(0);
            for (int i = 0; i < count && !rc; ++i) {
                dpslab_plan* pl = b->plans[i];
                pl->profiling = 0;
                rc = enqueue(pl, n[i], pos[i], q[i], phi ? phi[i] : nullptr, force ? force[i] : nullptr,
                             b->streams[i % S], kSolveAll);
                pl->last_n = n[i];
                launches += pl->launches;
            }
            join(0);
        }
        for (int w0 = 0, wave = 0; b->schedule == DPSLAB_BATCH_WAVES && w0 < count && !rc; w0 += S, ++wave) {
            const int w1 = std::min(count, w0 + S);
            fork(w0);
            for (int i = w0; i < w1 && !rc; ++i) {
                dpslab_plan* pl = b->plans[i];
                pl->profiling = 0;
                rc = enqueue(pl, n[i], pos[i], q[i], phi ? phi[i] : nullptr, force ? force[i] : nullptr,
                             b->streams[i % S], kSolveFront);
            }
            join(w0);
            // the wave's column stage: one launch per kind over all its systems' modes
            for (const auto& g : b->waves[wave]) {
                if (rc) break;
                if (g.kind == 0) k_column_batch<<<g.blocks, kColThreads, g.smem, st>>>(*g.arg);
                if (g.kind == 1) k_column_mixed_batch<<<g.blocks, kColThreadsM, g.smem, st>>>(*g.arg);
                if (g.kind == 2) column_tc_batch_kernel(g.tc_w, g.tc_r)<<<g.blocks, 64 * g.tc_w, g.smem, st>>>(*g.arg);
                ++launches;
                const cudaError_t le = cudaGetLastError();
                if (le != cudaSuccess) {
                    trace("batched column stage", le, __LINE__);
                    rc = DPSLAB_ERR_CUDA;
                }
            }
            fork(w0);
            for (int i = w0; i < w1 && !rc; ++i) {
                dpslab_plan* pl = b->plans[i];
                rc = enqueue(pl, n[i], pos[i], q[i], phi ? phi[i] : nullptr, force ? force[i] : nullptr,
                             b->streams[i % S], kSolveBack);
                pl->last_n = n[i];
                launches += pl->launches;
            }
            join(w0);
        }
        b->launches = launches;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        if (e != cudaSuccess) trace("cudaStreamEndCapture", e, __LINE__);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc ? rc : DPSLAB_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0);
        if (ie != cudaSuccess) {
            trace("cudaGraphInstantiate", ie, __LINE__);
            cudaGraphDestroy(g);
            b->exec = nullptr;
            return DPSLAB_ERR_CUDA;
        }
        b->graph = g;
        b->g_ptr = ptr;
        b->g_n.assign(n, n + count);
        b->g_schedule = b->schedule;
    }
    DPS_CUDA(cudaGraphLaunch(b->exec, st));
    DPS_CUDA(cudaEventRecord(b->out, st));
    DPS_CUDA(cudaStreamWaitEvent(caller, b->out, 0));
    DPS_CUDA(cudaStreamSynchronize(st));
    int first = DPSLAB_OK;
    for (int i = 0; i < count; ++i) {
        const int rc = collect(b->plans[i], U ? &U[i] : nullptr);
        if (rc && trace_on()) std::fprintf(stderr, "dpslab: batch system %d: code %d, status bits %d\n", i, rc, *b->plans[i]->h_status);
        if (status) status[i] = rc;
        if (rc && !first) first = rc;
    }
    return first;
}

extern "C" int64_t dpslab_batch_device_bytes(const dpslab_batch* b) { return b ? b->device_bytes : 0; }

extern "C" int dpslab_batch_last_launch_count(const dpslab_batch* b) { return b ? b->launches : 0; }

extern "C" int dpslab_batch_set_schedule(dpslab_batch* b, int schedule) {
    if (!b || (schedule != DPSLAB_BATCH_STREAMS && schedule != DPSLAB_BATCH_WAVES)) return DPSLAB_ERR_INVALID_ARG;
    b->schedule = schedule;
    return DPSLAB_OK;
}

extern "C" int dpslab_batch_schedule(const dpslab_batch* b) { return b ? b->schedule : DPSLAB_ERR_INVALID_ARG; }

extern "C" int dpslab_batch_autotune(dpslab_batch* b, const int64_t* n, const double* const* pos,
                                     const double* const* q, int reps, void* stream) {
    if (!b || !n || !pos || !q || reps < 1) return DPSLAB_ERR_INVALID_ARG;
    DPS_CUDA(cudaSetDevice(b->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DPS_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return DPSLAB_ERR_CUDA;
    }
    // median time of `reps` batch solves after one warm-up (which captures the graph)
    auto time_schedule = [&](int sched, double& out) -> int {
        b->schedule = sched;
        std::vector<double> t;
        for (int i = 0; i <= reps; ++i) {
            if (cudaEventRecord(e0, st) != cudaSuccess) return DPSLAB_ERR_CUDA;
            const int rc = dpslab_batch_solve(b, n, pos, q, nullptr, nullptr, nullptr, nullptr, stream);
            if (rc && rc != DPSLAB_ERR_NOT_NEUTRAL) return rc;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return DPSLAB_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (i) t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        out = t[t.size() / 2];
        return DPSLAB_OK;
    };
    const int cur = b->schedule;
    double t_cur = 0.0, t_other = 0.0;
    const int other = cur == DPSLAB_BATCH_STREAMS ? DPSLAB_BATCH_WAVES : DPSLAB_BATCH_STREAMS;
    int rc = time_schedule(cur, t_cur);
    if (!rc) rc = time_schedule(other, t_other);
    b->schedule = (!rc && t_other < 0.98 * t_cur) ? other : cur;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

extern "C" int dpslab_batch_destroy(dpslab_batch* b) {
    if (!b) return DPSLAB_ERR_INVALID_ARG;
    cudaSetDevice(b->device);
    batch_release(b);
    return DPSLAB_OK;
}
