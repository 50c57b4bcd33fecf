// Kernel parameter block and small device helpers of the FP64 solve.
#pragma once

#include <cuda_runtime.h>

#include "fft.cuh"
#include "internal.h"

namespace dps {

// Status bits written by kernels (read back once per solve).
enum : int {
    kStatusOutOfSlab = 1,
    kStatusNonFinite = 2,
    kStatusCapacity = 4,      // a bucketed-source buffer would overflow (not reachable within the bound)
    kStatusTimeout = 8,       // a bounded wait on the tensor-core pipeline gave up
    kStatusRejected = 16,     // every proposal of a Brownian-dynamics step left the slab
};

// The record types below are 16-byte aligned so that they move as 16-byte
// vector loads and stores (one L2 sector per 32-byte record, not eight).

// Interpolation window of one charge (mixed precision), Sec. 5.2.2 step 7:
// the same index rule as the spreading, evaluated once per charge in double;
// offsets of the first x and y points and z as a float pair.
struct __align__(16) IRec {
    float d0x, d0y;           // x_lo h_x - x, y_lo h_y - y
    float zhi, zlo;           // z = zhi + zlo
    int xlo, ylo;
    short sx, sy, j0, j1;     // support sizes, first and last z node
};

// A source of the mixed-precision spreading (float offsets and strength,
// z as a float pair), stored once per (tile, slab) block it touches.
struct __align__(16) SrcF {
    float d0x, d0y;           // x_lo h_x - x, y_lo h_y - y
    float zhi, zlo;           // z = zhi + zlo
    float q;                  // strength (image strengths for images)
    int xlo, ylo;             // first support index in x and y (unwrapped)
    unsigned pack;            // sx | sy << 6 | j0 << 12 | j1 << 21 | over << 30 | spread << 31
};

// Correction parameters of one k-mode for the node-value GEMM epilogue
// (mixed precision, normalised form of Eq. (inphisc)): the correction is
// iden (P (-(e1 - Gt e2)) + Q (e3 - Gb e4)) with e1 = e^{-kz}, e3 = e^{k(z-H)},
// e2 = e3 ekH, e4 = e1 ekH; corr = 0 for modes without one.
struct __align__(16) ColP {
    float2 P, Q;
    float k, ekH, iden;
    int corr;
};

// One spreading source (FP64) with its support precomputed: grid indices
// xlo..xlo+sx-1, ylo..ylo+sy-1 (unwrapped) and nodes j0..j1, offsets of the
// first x and y index from the source, strength, and whether it also feeds
// rho_o (a charge of C_over).
struct __align__(16) SrcRec {
    double z, q, d0x, d0y;
    int xlo, ylo, j0, j1;
    int sx, sy, over, pad;
};

// Everything a kernel needs, passed by value.
struct KP {
    // problem
    double Lx, Ly, H, eps, gw;
    double Gb, Gt;            // image factors (eps_w - eps)/(eps_w + eps); 1 for metal
    double cb, db, ct, dt;    // eps_w/(eps_w + eps), eps/(eps_w + eps) (metal: 1, 0)
    double tb, tt;            // tau_w = 2 eps/(eps_w + eps), Eq. (phibst)/(phitst)
    double rtb, rtt;          // (eps_w/eps) tau_w
    int metal_b, metal_t;
    // discretisation
    int nx, ny, nz, nxh;
    double hx, hy, HE, gt, xi, r_cut, a, b, Hbar, kmax;
    double s1norm;            // (2 pi g_t^2)^{-1/2}: one factor of Eq. (spreadkernelEw)
    double sigma2;            // (1/(2 xi))^2, 0 when xi = inf
    double inv_nxny;
    // near-field kernel widths: averaged (Eq. (GnearK)) and pointwise (Eq. (Gnear))
    double na1, na2, pa1, pa2;   // a2 = 0 encodes "infinite" (xi = 0), a1 == a2 disables
    int near_on;
    // Narrow widths (1/a2 close to 1/a1): the averaged kernel as
    // (2/sqrt(pi)) int_{1/a2}^{1/a1} e^{-r^2 s^2} ds by 4-point Gauss-Legendre,
    // nodes gq_s and weights gq_w on that interval (used in float)
    int near_quad;
    float gq_s[4], gq_w[4];
    // float copies of the scalars the mixed-precision kernels use per element
    struct {
        float kxs, kys;                   // 2 pi/Lx, 2 pi/Ly
        float H, HE, Hbar, sz;            // sz = 2/Hbar (d/dz of the scaled coordinate)
        float scale;                      // -(Hbar/2)^2/eps (right-hand side of Eq. (blocksys))
        float Gb, Gt, cb, db, ct, dt, tb, tt, rtb, rtt;
        float sigma2;
        float hx, hy, ig2, s1norm;        // grid steps, 1/(2 g_t^2), (2 pi g_t^2)^{-1/2}
        float a;                          // lower end of the Chebyshev interval
    } f;
    // charges
    int n;
    const double* pos;
    const double* q;
    double4_32a* part;            // sanitised (x, y, z, q)
    // grids, in the plan's grid precision R (double for DPSLAB_FP64, float
    // for DPSLAB_MIXED)
    void* rho;                // R [2][nz][ny][nx]
    void* spec;               // complex R [2][nz][ny][nxh]
    void* specB;              // complex R [nz][ny][nxh]
    void* fields;             // R4 [nz][ny][nx] (phi, Ex, Ey, Ez)
    int mixed;
    // tables
    const double* zn;
    const double* wz;
    const double* cft;        // split forward transform, input-major (see Tables)
    const double *tie, *tio;  // split inverse transform, [n/2][a]
    const double *j2l, *j2d, *j2u, *u1, *u2, *v1, *v2, *t0, *tH, *wg;
    const double2* twx;
    const double2* twy;
    const float2* twx32;      // the same twiddles rounded to float
    const float2* twy32;
    // float copies of the column tables (mixed precision)
    const float* zn32;        // z_j rounded to float
    const float* hinv32;      // 1/(2n), n >= 1 (integration recurrence)
    const float* znlo32;      // z_j - zn32[j] (z_j as a float pair)
    const float* wzh32;       // Clenshaw-Curtis weight times h_x h_y
    const float *cft32, *tie32, *tio32, *j2l32, *j2d32, *j2u32, *u132, *u232, *v132, *v232, *t032, *tH32, *wg32;
    int radx[kMaxStages], rady[kMaxStages];
    int nradx, nrady;
    // particle outputs
    double4_32a* far;             // [n] (phibar, Ebar)
    double4_32a* nearv;           // [n]
    // spreading tiles: 16 x 16 xy grid points by `slab` z nodes; the sources
    // (charges and their images) are counting-sorted into (slab, tile) buckets
    int ntx, nty, ntiles, tile_r, slab, nslabs, nbuckets, supx, supy;
    int* tile_count;          // per bucket
    int* tile_start;          // nbuckets + 1
    int* tile_fill;
    struct SrcRec* srcs;      // bucketed source records
    SrcF* srcsf;              // the same storage, mixed-precision records
    size_t src_cap;           // capacity of srcsf in records
    // cell list
    int ncx, ncy, ncz, ncells;
    double cwx, cwy, cwz;     // cell widths
    int* cell_of;
    int* cell_count;
    int* cell_start;          // ncells + 1
    int* cell_fill;
    double4_32a* sorted;
    float4* sorted_rel;       // float offsets from the cell corner, and q (mixed near field)
    IRec* irec;               // [n] interpolation windows in cell-list order (mixed)
    SrcF* srcs_tmp;           // [3n] sources of each charge before bucketing, same order (mixed)
    ColP* colp;               // [ny nxh] correction parameters per mode (tensor-core z transforms)
    double* zcol;             // [2 nz + 1] mixed: the k = 0 column from k_column_zero (y, y', gauge term)
    // J^T t0, J^T J^T t0, J^T tH, J^T J^T tH (J: Appendix-A integration,
    // y' = J y'' + d e0, y = J y' + c e0), float: wall values from y'' directly
    const float *jt0_32, *jjt0_32, *jtH_32, *jjtH_32;
    const double4_32a* mtab;  // [ny nxh] mixed: per mode k, e^{-kH}, 1/den, -(1 - Gt e^{-2kH})/den (k only: no correction)
    const unsigned short* zimg_fwd;   // split bf16 images of the z transforms (tensor cores)
    // mixed, tensor-core form, per node: bit 0 where rho_o can be non-zero
    // (within H_E of a charge of C_over: z_j in [-H_E, 3 H_E] or
    // [H - 3 H_E, H + H_E]), bit 1 where the interpolation reads the fields
    // (z_j in [-H_E, H + H_E]); null: every node has both. rho_o is neither
    // stored, transformed in x and y, nor read by the forward z transform
    // without bit 0; the inverse transforms neither form nor store the
    // fields without bit 1.
    const unsigned char* node_mask;
    // mixed, tensor-core form: rho_o's Chebyshev coefficients come from its
    // node values at the o_pairs node pairs (a, m - a) it can reach, formed
    // in the column kernel instead of the tensor-core transform: o_pair[p] =
    // a (a <= m - a), o_fwd[p][n] = the forward transform's entry for node a
    // and coefficient n, applied to v_a + v_{m-a} for even n and
    // v_a - v_{m-a} for odd n. o_pairs = 0: the z transform handles rho_o.
    int o_pairs;
    const int* o_pair;
    const float* o_fwd;
    const unsigned short* zimg_inv;
    int* sorted_idx;
    // reductions
    double* part_gauge_far;   // one per column block
    double* part_gauge_near;  // one per charge block
    double* part_u;           // one per charge block
    double* part_q;           // [2 * nblocks]: sum q, sum |q|
    double* scal;             // [16]: B, A_i, phi_f0, phi_n0, U, sumq, sumabsq, k=0 far potential at
                              // z = 0 and z = H (unnormalised; wall charges), spare
    // wall charge densities (Eq. (rho)): their xy transforms, the potential
    // grid of their k != 0 correction, per-charge terms of the wall energy
    int sigma_on;
    const double2* sig_hat;   // [2][ny nxh]: sigma_b, sigma_t transforms (unnormalised)
    const void* sig_grid;     // R [nz][ny][nx]: correction driven by the wall charges alone
    double* wall_phi;         // [n] phibar of that correction at each charge
    double* part_wall;        // [3 * nblocks]: q phibar_sigma, near planar sums at z = 0, H
    const double* wgH;        // gauge weights at z = H
    double sig_Qb, sig_Qt;    // total wall charges int sigma dx dy
    double sig_self;          // 1/2 int sigma phi_sigma over both walls (k != 0)
    // Brownian dynamics scratch: steric forces, proposal, proposed noise [n][3]; flags per retry
    double *bd_steric, *bd_prop, *bd_wnew;
    int* bd_flags;
    int* status;
    long long zspin;          // polls of each bounded wait in the tensor-core z transforms
    int n_col_blocks, n_charge_blocks;
    // user outputs
    double* out_phi;
    double* out_force;
};

// row (of the 2 nz ny rows of both densities) of rho_o at a node it cannot reach
__device__ __forceinline__ bool o_row_zero(const KP& kp, int row) {
    const int nzy = kp.nz * kp.ny;
    return kp.node_mask && row >= nzy && !(kp.node_mask[(row - nzy) / kp.ny] & 1);
}

// row (of the nz ny rows of a field grid) at a node the interpolation never reads
__device__ __forceinline__ bool f_row_skip(const KP& kp, int row) {
    return kp.node_mask && !(kp.node_mask[row / kp.ny] & 2);
}
// rows r0 .. r0 + P - 1 (P <= 64) skipped by f_row_skip: bit p for row r0 + p
// (rows past nrows count as skipped)
__device__ __forceinline__ unsigned long long f_rows_skip(const KP& kp, int r0, int P, int nrows) {
    if (!kp.node_mask) {
        unsigned long long m = 0ull;
        for (int p = 0; p < P; ++p)
            if (r0 + p >= nrows) m |= 1ull << p;
        return m;
    }
    unsigned long long m = 0ull;
    for (int p = 0; p < P; ++p)
        if (r0 + p >= nrows || f_row_skip(kp, r0 + p)) m |= 1ull << p;
    return m;
}

template <class R> struct Prec;
template <> struct Prec<double> {
    using C = double2;
    using V4 = double4_32a;
    static __device__ __forceinline__ V4 v4(double a, double b, double c, double d) { return make_double4_32a(a, b, c, d); }
};
template <> struct Prec<float> {
    using C = float2;
    using V4 = float4;
    static __device__ __forceinline__ V4 v4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double derf(double x) { return erf(x); }
__device__ __forceinline__ float derf(float x) { return erff(x); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

__device__ __forceinline__ double np_mod(double x, double L) {
    // numpy float remainder: fmod, then shifted into the sign of L (a point
    // already in [0, L) is its own remainder)
    if (x >= 0.0 && x < L) return x;
    double r = fmod(x, L);
    if (r != 0.0 && r < 0.0) r += L;
    return r;
}

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

// erf(r/a)/r and (1/r) d/dr[erf(r/a)/r]; series for r < 1e-3 g_w (end of Sec. 3.2)
template <class R>
__device__ __forceinline__ void erf_over_r(R r, R a, bool small, R& val, R& der) {
    const R x = r / a;
    const R c = R(1.1283791670955126) / a;   // 2/(sqrt(pi) a)
    if (small) {
        const R x2 = x * x;
        val = c * (R(1) - x2 / R(3) + x2 * x2 / R(10) - x2 * x2 * x2 / R(42));
        der = c * (R(-2) / (R(3) * a * a) + R(4) * x2 / (R(10) * a * a) - R(6) * x2 * x2 / (R(42) * a * a));
    } else {
        const R e = derf(x);
        val = e / r;
        der = (-e / (r * r) + c * dexp(-x * x) / r) / r;
    }
}

// near-field kernel value and (1/r) dG/dr for widths (a1, a2); a2 == 0 means infinite
template <class R>
__device__ __forceinline__ void near_kernel(R r, R a1, R a2, R gw, R eps, R& g, R& d) {
    const bool small = r < R(1e-3) * gw;
    R v1, d1, v2 = 0, d2 = 0;
    erf_over_r<R>(r, a1, small, v1, d1);
    if (a2 > R(0)) erf_over_r<R>(r, a2, small, v2, d2);
    const R s = R(1) / (R(12.566370614359172) * eps);   // 1/(4 pi eps)
    g = (v1 - v2) * s;
    d = (d1 - d2) * s;
}

// Averaged near-field kernel in float without cancellation (narrow widths):
// Gbar = (1/(4 pi eps)) (2/sqrt(pi)) int e^{-r^2 s^2} ds and
// (1/r) dGbar/dr = -(1/(4 pi eps)) (4/sqrt(pi)) int s^2 e^{-r^2 s^2} ds over
// s in [1/a2, 1/a1]; the erf difference of Eq. (GnearK) written as an integral.
__device__ __forceinline__ void near_kernel_quad(const KP& kp, float r, float& g, float& d) {
    const float r2 = r * r;
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float s = kp.gq_s[i];
        const float e = kp.gq_w[i] * expf(-r2 * s * s);
        a += e;
        b += s * s * e;
    }
    const float c = float(1.0 / (12.566370614359172 * kp.eps));
    g = 1.1283791670955126f * a * c;
    d = -2.2567583341910252f * b * c;
}

}  // namespace dps
