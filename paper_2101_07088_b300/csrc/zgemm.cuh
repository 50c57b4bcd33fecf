// z-direction Chebyshev transforms as tensor-core GEMMs (sm_103a, tcgen05).
//
// Sec. 5.2.2 steps 3 and 6 apply one dense Nz x Nz matrix to every k-mode
// column: coefficients from node values (the DCT-I form of the extrema-grid
// transform) and node values from coefficients (T_n(s_j) = cos(pi n j/m)).
// With the columns of a spectrum plane as the N dimension this is
//     D[128 x N] = A[128 x 128] . B[128 x N]      (rows and K padded to 128)
// over N = 2 ny (nx/2+1) real columns per plane (real and imaginary parts).
//
// Precision: A and B are split into three bf16 pieces each, x = x1 + x2 + x3,
// and the six products with piece orders summing to at most 4 (11, 12, 21,
// 13, 22, 31) are kept; the dropped terms are below 2^-24 of the largest
// entry. The tensor core adds into its FP32 accumulator with truncation (a
// bias toward zero of up to one ulp per K step), which a plain split turns
// into a systematic error of ~1e-6. Hence x1 lies on a fixed-point grid,
// rint(x 128/s) s/128, with s the power of two above the largest |x| of the
// row of A (host) or of the column of B (per tile, here): x1 128/s is an
// integer of at most 8 bits, so every partial sum of the dominant product 11
// is an integer multiple of one unit below 2^21 units, exact in FP32 - it is
// never truncated. It has its own accumulator; the five small products share
// a second one (their truncation is 2^-7 smaller), and the two are added on
// the CUDA cores in round-to-nearest. x2 and x3 are bf16 roundings of the rest.
//
// One persistent CTA of 512 threads per SM keeps A (three pieces, 96 KB) in
// shared memory and loops over N tiles of 128 columns:
//   1. the threads split the tile's values (held in registers, loaded during
//      the previous tile's MMAs, 16-byte loads of 4 columns x 8 rows per
//      thread) into the three bf16 B pieces, canonical K-major layout
//      (8 x 16-byte core matrices, no swizzle);
//   2. one thread issues the 6 x 8 tcgen05.mma (M=128, N=128, K=16,
//      kind::f16, bf16 inputs, FP32 accumulators) and commits them to an
//      mbarrier; meanwhile the threads load the next tile;
//   3. each warp reads its quarter of the accumulator lanes, 32 columns, with
//      tcgen05.ld, adds the two accumulators and stores the rows through an
//      epilogue functor.
// The waits on the MMAs and on the bulk copies are bounded (`spin` polls);
// on a timeout the kernel records kStatusTimeout, stops, waits for the work
// still in flight (bounded by kZSpinLimit polls, whatever `spin` is) and
// frees its tensor memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "kernels.cuh"

namespace dps {

constexpr int kZK = 128;          // K and M of the GEMM (Nz padded)
constexpr int kZN = 128;          // N tile (floats)
constexpr int kZThreads = 512;
constexpr int kZPieceA = kZK * kZK;         // bf16 elements per A piece
// B row groups (8 columns, all K) 2064 B apart instead of 2048: a warp's
// 16-byte stores into 16 groups then fall on different banks
constexpr int kZSboB = 2048 + 16;           // bytes between B row groups
constexpr int kZPieceB = (kZN / 8) * (kZSboB / 2);   // bf16 elements per B piece
constexpr size_t kZSmemA = 3 * size_t(kZPieceA) * 2;
constexpr size_t kZSmemB = 3 * size_t(kZPieceB) * 2;
constexpr int kZOStride = kZN + 4;          // staged output row stride (16-byte rows, conflict-free)
constexpr int kZORows = 32;                 // rows of the single-block path's staging area
constexpr size_t kZSmemO = size_t(kZORows) * kZOStride * 4;
constexpr size_t kZSmem = kZSmemA + kZSmemB + 64 + kZSmemO;
constexpr int kZRows = 8;                   // rows per thread and tile (4 columns each)
constexpr int kZGroups = kZK / kZRows;      // row groups of a tile
constexpr long kZSpinLimit = 1L << 26;      // polls of an mbarrier before giving up
static_assert(kZThreads == (kZN / 4) * kZGroups, "one (column quad, row group) per thread");
static_assert(kZMaxNz <= 2 * kZBlock, "at most two K blocks (held in registers)");

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N)
// byte offsets >> 4, descriptor version 1 (bits 46-47), no swizzle
__device__ __forceinline__ uint64_t zdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((saddr & 0x3FFFF) >> 4) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

// instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// bf16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t zidesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait of at most `limit` polls; false on timeout (at once for limit 0)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = kZSpinLimit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// one-dimensional bulk copy global -> shared (both 16-byte aligned, bytes a
// multiple of 16) that signals `bar` with its byte count
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
// 16 consecutive 32-bit accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x = x1 + x2 + x3: x1 = rint(x q) / q on the fixed-point grid of step 1/q
// (q = 128/s, a power of two), x2, x3 bf16 roundings of the rest (each
// residual exact in FP32)
__device__ __forceinline__ void split3(float x, float q, float iq, __nv_bfloat16& a, __nv_bfloat16& b,
                                       __nv_bfloat16& c) {
    const float x1 = rintf(x * q) * iq;
    a = __float2bfloat16_rn(x1);
    const float r1 = x - x1;
    b = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b);
    c = __float2bfloat16_rn(r2);
}

// 8 values at K entries k0..k0+7 of column n, three pieces, one 16-byte
// store each. The same split as split3, two values at a time: x1 has at
// most 8 significant bits, so its bf16 is the upper half of the float
// (exact), and two halves pack with one byte permutation; the other two
// pieces are rounded in pairs.
__device__ __forceinline__ void put8(unsigned short* sB, int n, int k0, const float* x, float q, float iq) {
    uint4 w1, w2, w3;
    uint32_t* v1 = &w1.x;
    uint32_t* v2 = &w2.x;
    uint32_t* v3 = &w3.x;
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
        const float x1a = rintf(x[i] * q) * iq, x1b = rintf(x[i + 1] * q) * iq;
        v1[i / 2] = __byte_perm(__float_as_uint(x1a), __float_as_uint(x1b), 0x7632);
        const float r1a = x[i] - x1a, r1b = x[i + 1] - x1b;
        const __nv_bfloat162 b = __floats2bfloat162_rn(r1a, r1b);
        const __nv_bfloat162 c = __floats2bfloat162_rn(r1a - __low2float(b), r1b - __high2float(b));
        v2[i / 2] = *reinterpret_cast<const uint32_t*>(&b);
        v3[i / 2] = *reinterpret_cast<const uint32_t*>(&c);
    }
    const int e = (n >> 3) * (kZSboB / 2) + (k0 >> 3) * 64 + (n & 7) * 8;   // canonical layout, padded row groups
    *reinterpret_cast<uint4*>(sB + e) = w1;
    *reinterpret_cast<uint4*>(sB + kZPieceB + e) = w2;
    *reinterpret_cast<uint4*>(sB + 2 * kZPieceB + e) = w3;
}

// mask1 (optional, Nz bytes): rows of plane 1 to read where bit 0 is set;
// the others are zero (rho_o at the nodes it cannot reach) and are not
// loaded. smask (optional, Nz bytes): output rows to form and store where
// bit 1 is set (the nodes the interpolation reads); the others are left as
// they are.
// The GEMM over nplanes planes of rows (= Nz) x ncols floats (row stride ld,
// plane stride pstride floats; ld and the plane base multiples of 4 floats),
// written back in place. A image: three pieces, zimg_index layout.
// epi(plane, row, col0, v[32], nvalid) may change the 32 outputs of row `row`
// from column col0 before they are stored (the tile is staged in shared
// memory so that each warp store writes 512 contiguous bytes of one row).
static_assert(size_t(kZK) * kZOStride * 4 <= kZSmemB, "staged outputs fit the B pieces");
// prep(plane, col0) runs on every thread once per tile while the MMAs are in
// flight (before the barrier that precedes the epilogue): it may stage
// per-tile data in shared memory for epi.
// nblk = 1 (Nz <= 128): A stays in shared memory for all tiles and the next
// tile's values load during the MMAs. nblk = 2 (128 < Nz <= 256): rows and K
// come in two blocks of 128; each thread holds its 4 columns' 16 values of
// the tile (8 per K block), so the column maxima over all K (one fixed-point
// grid per column for the exact product) need no second read. For each K
// block the values are split into B and, for each row block, that block of
// A is staged by one bulk copy and its MMAs accumulate into the row block's
// two accumulators (four in all, the whole 512 columns of tensor memory).
// The outputs are written, in place, after every K row of the tile has been
// read; the next tile's values load from the last split on.
template <bool kRead1, class Prep, class Epi>
__device__ __forceinline__ void zgemm_run(const unsigned short* __restrict__ aimg, float* base, int nplanes,
                                          size_t pstride, int rows, int ncols, size_t ld, int* status, Prep prep,
                                          Epi epi, int nblk, long long spin, const unsigned char* mask1 = nullptr,
                                          const unsigned char* smask = nullptr) {
    extern __shared__ __align__(1024) unsigned char zsm[];
    unsigned short* sA = reinterpret_cast<unsigned short*>(zsm);
    unsigned short* sB = reinterpret_cast<unsigned short*>(zsm + kZSmemA);
    uint64_t* bar = reinterpret_cast<uint64_t*>(zsm + kZSmemA + kZSmemB);
    uint64_t* abar = bar + 1;                   // bulk copies of the A blocks (nblk > 1)
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 2);
    __shared__ int s_abort;
    // column maxima: per (column offset j of a quad, row group, quad) and
    // reduced over the row groups (transposed so that both passes are
    // conflict-free)
    __shared__ float s_cmT[4][kZGroups][kZN / 4];
    __shared__ float s_amax[4][kZN / 4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_per_plane = (ncols + kZN - 1) / kZN;
    const int ntiles = nplanes * tiles_per_plane;
    // this thread's 4 columns (4 cq .. 4 cq + 3) and 8 rows (8 g .. 8 g + 7)
    const int cq = tid & (kZN / 4 - 1), g = tid / (kZN / 4), r0 = g * kZRows;
    // rows plane 1 reads (mask1 bit 0) and output rows formed and stored
    // (smask bit 1): bit r % 32 of word r / 32 (filled by warp 0 below)
    __shared__ unsigned s_read1[2 * kZBlock / 32], s_store[2 * kZBlock / 32];
    if (warp == 0) {
        for (int i = 0; i < 2 * kZBlock / 32; ++i) {
            const int r = 32 * i + lane;
            const unsigned rd = __ballot_sync(0xffffffffu, !mask1 || (r < rows && (mask1[r] & 1)));
            const unsigned sv = __ballot_sync(0xffffffffu, !smask || (r < rows && (smask[r] & 2)));
            if (lane == 0) {
                s_read1[i] = rd;
                s_store[i] = sv;
            }
        }
    }
    auto stored = [&](int r) { return (s_store[r >> 5] >> (r & 31)) & 1u; };
    // the largest |entry| of this thread's four columns over all rows of the
    // tile, from each thread's partial maxima cm
    auto colmax = [&](const float* cm, float* amax) {
#pragma unroll
        for (int j = 0; j < 4; ++j) s_cmT[j][g][cq] = cm[j];
        __syncthreads();
        if (tid < kZN) {
            const int j = tid / (kZN / 4), c = tid & (kZN / 4 - 1);
            float m = 0.f;
#pragma unroll
            for (int i = 0; i < kZGroups; ++i) m = fmaxf(m, s_cmT[j][i][c]);
            s_amax[j][c] = m;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) amax[j] = s_amax[j][cq];
    };

    auto stage_a = [&](int rb, int kb) {     // block (rb, kb) of the image into shared memory
        const uint4* src = reinterpret_cast<const uint4*>(aimg + zimg_block(rb, kb, nblk, 0));
        uint4* dst = reinterpret_cast<uint4*>(sA);
        for (int i = tid; i < int(kZSmemA / 16); i += blockDim.x) dst[i] = src[i];
    };
    // tensor memory: nblk = 1 keeps two tiles' accumulators (the epilogue of
    // one runs while the MMAs of the next are in flight); nblk = 2 the four
    // accumulators of one tile
    const uint32_t tcols = 4u * kZN;
    float* sO = reinterpret_cast<float*>(zsm + kZSmemA + kZSmemB + 64);   // nblk = 1 staging
    if (nblk == 1) stage_a(0, 0);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(abar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    // kRead1: which of this thread's rows plane 1 reads (bit kb 8 + i: row
    // kb 128 + r0 + i; r0 is a multiple of 8, so each block's 8 rows lie in
    // one mask word)
    unsigned rows1 = 0xffffu;
    if (kRead1)
        rows1 = ((s_read1[r0 >> 5] >> (r0 & 31)) & 0xffu) | (((s_read1[(kZBlock + r0) >> 5] >> (r0 & 31)) & 0xffu) << 8);

    float4 rv[kZRows];
    auto load = [&](int t, int kb) {         // K rows kb*128 + r0 .. + 7 of tile t
        const int plane = t / tiles_per_plane, c0 = (t - plane * tiles_per_plane) * kZN;
        const int c = c0 + 4 * cq;
        const float* src = base + size_t(plane) * pstride + c;
        const int rb0 = kb * kZBlock + r0;
        const unsigned rm = (kRead1 && plane == 1) ? rows1 >> (kb * kZRows) : 0xffu;
#pragma unroll
        for (int i = 0; i < kZRows; ++i) {
            const int r = rb0 + i;
            rv[i] = (r < rows && c < ncols && ((rm >> i) & 1u)) ? __ldg(reinterpret_cast<const float4*>(src + size_t(r) * ld))
                                                                : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };

    uint32_t ph = 0u, aph = 0u;
    bool pend = false, apend = false;
    if (nblk > 1) {
        // both K blocks of the tile in registers: rv rows r0.., rw rows 128 + r0..
        float4 rw[kZRows];
        auto load2 = [&](int t) {
            load(t, 0);
            const int plane = t / tiles_per_plane, c0 = (t - plane * tiles_per_plane) * kZN;
            const int c = c0 + 4 * cq;
            const float* src = base + size_t(plane) * pstride + c;
            const int rb1 = kZBlock + r0;
            const unsigned rm = (kRead1 && plane == 1) ? rows1 >> kZRows : 0xffu;
#pragma unroll
            for (int i = 0; i < kZRows; ++i) {
                const int r = rb1 + i;
                rw[i] = (r < rows && c < ncols && ((rm >> i) & 1u)) ? __ldg(reinterpret_cast<const float4*>(src + size_t(r) * ld))
                                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        if (int(blockIdx.x) < ntiles) load2(blockIdx.x);
        for (int t = blockIdx.x; t < ntiles && !s_abort; t += gridDim.x) {
            const int plane = t / tiles_per_plane, c0 = (t - plane * tiles_per_plane) * kZN;
            const int w = min(kZN, ncols - c0);
            // each column's largest |entry| over all K: one fixed-point grid
            // per column for the exact product
            float am[4];
            {
                float cm[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < kZRows; ++i) {
                    cm[0] = fmaxf(cm[0], fmaxf(fabsf(rv[i].x), fabsf(rw[i].x)));
                    cm[1] = fmaxf(cm[1], fmaxf(fabsf(rv[i].y), fabsf(rw[i].y)));
                    cm[2] = fmaxf(cm[2], fmaxf(fabsf(rv[i].z), fabsf(rw[i].z)));
                    cm[3] = fmaxf(cm[3], fmaxf(fabsf(rv[i].w), fabsf(rw[i].w)));
                }
                colmax(cm, am);
            }
            float qv[4], iqv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float amax = am[j];
                int e = 0;
                if (amax > 0.f) frexpf(amax, &e);
                qv[j] = ldexpf(1.f, 7 - e);
                iqv[j] = ldexpf(1.f, e - 7);
            }
            for (int kb = 0; kb < nblk && !s_abort; ++kb) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float x[kZRows];
#pragma unroll
                    for (int i = 0; i < kZRows; ++i) {
                        const float4 a = kb == 0 ? rv[i] : rw[i];
                        x[i] = j == 0 ? a.x : j == 1 ? a.y : j == 2 ? a.z : a.w;
                    }
                    put8(sB, 4 * cq + j, r0, x, qv[j], iqv[j]);
                }
                // the last K block is in B: the next tile's values load while
                // the remaining copies, MMAs and the epilogue run
                if (kb == nblk - 1 && t + int(gridDim.x) < ntiles) load2(t + gridDim.x);
                for (int rb = 0; rb < nblk; ++rb) {
                    // block (rb, kb) of A by one bulk copy (the previous MMAs,
                    // which read sA, have completed)
                    if (tid == 0) {
                        mbar_expect_tx(abar, uint32_t(kZSmemA));
                        bulk_g2s(sA, aimg + zimg_block(rb, kb, nblk, 0), uint32_t(kZSmemA), abar);
                        apend = true;
                        if (mbar_wait(abar, aph, spin)) apend = false;
                        else s_abort = 1;
                    }
                    fence_async_smem();
                    __syncthreads();
                    if (s_abort) break;
                    aph ^= 1u;
                    if (tid == 0) {
                        tc_fence_after();
                        constexpr uint32_t idesc = zidesc(kZK, kZN);
                        const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
                        const uint32_t d0 = tmem + uint32_t(rb * 2 * kZN);
                        const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
                        for (int qd = 0; qd < 6; ++qd)
#pragma unroll
                            for (int s8 = 0; s8 < kZK / 16; ++s8) {
                                const uint64_t ad = zdesc(a0 + uint32_t(pa[qd]) * kZPieceA * 2 + uint32_t(s8) * 256u, 128u, 2048u);
                                const uint64_t bd = zdesc(b0 + uint32_t(pb[qd]) * kZPieceB * 2 + uint32_t(s8) * 256u, 128u, kZSboB);
                                const bool first = kb == 0 && s8 == 0 && qd <= 1;
                                tc_mma(d0 + (qd == 0 ? 0u : uint32_t(kZN)), ad, bd, idesc, first ? 0u : 1u);
                            }
                        tc_commit(bar);
                    }
                    pend = true;
                    if (tid == 0 && !mbar_wait(bar, ph, spin)) s_abort = 1;
                    __syncthreads();
                    if (!s_abort) {
                        ph ^= 1u;
                        pend = false;
                    }
                    tc_fence_after();
                    if (s_abort) break;
                }
            }
            if (s_abort) break;
            prep(plane, c0);
            __syncthreads();
            // epilogue per row block: warp = TMEM lane quarter x 32 columns
            const int qtr = warp & 3, cc = (warp >> 2) * 32;
            const int r = qtr * 32 + lane;
            const int wv = min(32, w - cc);
            float* O = reinterpret_cast<float*>(sB);
            for (int rb = 0; rb < nblk; ++rb) {
                const int rg = rb * kZBlock + r;
                const uint32_t lb = tmem + (uint32_t(qtr * 32) << 16) + uint32_t(rb * 2 * kZN + cc);
                float v[32], u[16];
#pragma unroll
                for (int h = 0; h < 32; h += 16) {
                    tc_ld16(lb + uint32_t(h), v + h);
                    tc_ld16(lb + uint32_t(kZN + h), u);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[h + i] += u[i];
                }
                if (rg < rows && wv > 0 && stored(rg)) epi(plane, rg, c0 + cc, v, wv);
#pragma unroll
                for (int i = 0; i < 32; i += 4)
                    *reinterpret_cast<float4*>(O + r * kZOStride + cc + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                __syncthreads();
                float* dst = base + size_t(plane) * pstride + c0 + 4 * lane;
                if (4 * lane < w) {
                    for (int rr = warp; rr < kZBlock && rb * kZBlock + rr < rows; rr += kZThreads / 32)
                        if (stored(rb * kZBlock + rr))
                            __stcs(reinterpret_cast<float4*>(dst + size_t(rb * kZBlock + rr) * ld),
                                   *reinterpret_cast<const float4*>(O + rr * kZOStride + 4 * lane));
                }
                __syncthreads();
            }
            tc_fence_before();
            fence_async_smem();
            __syncthreads();
        }
    }
    // nblk = 1. Per tile t: split the values into B, issue the MMAs into
    // accumulator buffer (i & 1), prefetch the next tile's values, then run
    // the epilogue of tile t - 1 from the other buffer while those MMAs are
    // in flight, and wait for them (B is then free for the next split).
    auto epilogue = [&](int t, uint32_t tb) {
        const int plane = t / tiles_per_plane, c0 = (t - plane * tiles_per_plane) * kZN;
        const int w = min(kZN, ncols - c0);
        // warp: TMEM lane quarter (warp % 4) = rows, 32 columns ((warp / 4) * 32)
        const int qtr = warp & 3, cc = (warp >> 2) * 32;
        const int r = qtr * 32 + lane;
        const uint32_t lb = tb + (uint32_t(qtr * 32) << 16) + uint32_t(cc);
        float v[32], u[16];
#pragma unroll
        for (int h = 0; h < 32; h += 16) {
            tc_ld16(lb + uint32_t(h), v + h);
            tc_ld16(lb + uint32_t(kZN + h), u);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[h + i] += u[i];
        }
        const int wv = min(32, w - cc);
        if (r < rows && wv > 0 && stored(r)) epi(plane, r, c0 + cc, v, wv);
        // staged a quarter (32 rows) at a time, then stored whole rows: warp w
        // stores rows w and w + 16 of the quarter, lane l columns 4l .. 4l + 3
        float* dst = base + size_t(plane) * pstride + c0 + 4 * lane;
        for (int q = 0; q < kZK / kZORows; ++q) {
            if (qtr == q) {
#pragma unroll
                for (int i = 0; i < 32; i += 4)
                    *reinterpret_cast<float4*>(sO + lane * kZOStride + cc + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
            __syncthreads();
            if (4 * lane < w) {
                for (int rr = warp; rr < kZORows; rr += kZThreads / 32) {
                    const int row = q * kZORows + rr;
                    if (row < rows && stored(row))
                        __stcs(reinterpret_cast<float4*>(dst + size_t(row) * ld),
                               *reinterpret_cast<const float4*>(sO + rr * kZOStride + 4 * lane));
                }
            }
            __syncthreads();
        }
    };
    int prev_t = -1;
    uint32_t prev_buf = 0u;
    if (nblk == 1 && int(blockIdx.x) < ntiles) load(blockIdx.x, 0);
    for (int t = blockIdx.x, it = 0; nblk == 1 && t < ntiles; t += gridDim.x, ++it) {
        const uint32_t buf = tmem + uint32_t((it & 1) * 2 * kZN);
        // per column, the largest |entry| (fixed-point scale of piece 1), then
        // the split into the three pieces at K entries r0 .. r0 + 7
        float cm[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < kZRows; ++i) {
            cm[0] = fmaxf(cm[0], fabsf(rv[i].x));
            cm[1] = fmaxf(cm[1], fabsf(rv[i].y));
            cm[2] = fmaxf(cm[2], fabsf(rv[i].z));
            cm[3] = fmaxf(cm[3], fabsf(rv[i].w));
        }
        float am[4];
        colmax(cm, am);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = 4 * cq + j;
            const float amax = am[j];
            int e = 0;
            if (amax > 0.f) frexpf(amax, &e);
            const float q = ldexpf(1.f, 7 - e), iq = ldexpf(1.f, e - 7);   // 128/s, s/128 with s = 2^e > amax
            float x[kZRows];
#pragma unroll
            for (int i = 0; i < kZRows; ++i) x[i] = j == 0 ? rv[i].x : j == 1 ? rv[i].y : j == 2 ? rv[i].z : rv[i].w;
            put8(sB, n, r0, x, q, iq);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            constexpr uint32_t idesc = zidesc(kZK, kZN);
            const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
            const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
            for (int qd = 0; qd < 6; ++qd)
#pragma unroll
                for (int s8 = 0; s8 < kZK / 16; ++s8) {
                    const uint64_t ad = zdesc(a0 + uint32_t(pa[qd]) * kZPieceA * 2 + uint32_t(s8) * 256u, 128u, 2048u);
                    const uint64_t bd = zdesc(b0 + uint32_t(pb[qd]) * kZPieceB * 2 + uint32_t(s8) * 256u, 128u, kZSboB);
                    const bool first = s8 == 0 && qd <= 1;      // first K step of either accumulator
                    tc_mma(buf + (qd == 0 ? 0u : uint32_t(kZN)), ad, bd, idesc, first ? 0u : 1u);
                }
            tc_commit(bar);
        }
        pend = true;
        // the next tile's values, while the tensor cores work
        if (t + int(gridDim.x) < ntiles) load(t + gridDim.x, 0);
        if (prev_t >= 0) {
            const int pplane = prev_t / tiles_per_plane;
            prep(pplane, (prev_t - pplane * tiles_per_plane) * kZN);
            __syncthreads();
            tc_fence_after();
            epilogue(prev_t, prev_buf);
        }
        // one thread polls the MMA barrier (polls from every warp would
        // compete with the loads for the memory pipes); the rest wait here
        if (tid == 0 && !mbar_wait(bar, ph, spin)) s_abort = 1;
        tc_fence_before();
        __syncthreads();
        if (s_abort) break;
        ph ^= 1u;
        pend = false;
        tc_fence_after();
        prev_t = t;
        prev_buf = buf;
    }
    if (nblk == 1 && prev_t >= 0 && !s_abort) {
        const int pplane = prev_t / tiles_per_plane;
        prep(pplane, (prev_t - pplane * tiles_per_plane) * kZN);
        __syncthreads();
        tc_fence_after();
        epilogue(prev_t, prev_buf);
    }
    if (s_abort && tid == 0) {
        atomicOr(status, kStatusTimeout);
        if (pend) mbar_wait(bar, ph);
        if (apend) mbar_wait(abar, aph);     // a bulk copy of A still in flight
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

}  // namespace dps
