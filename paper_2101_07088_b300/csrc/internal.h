// Internal declarations shared by the planner (host C++) and the CUDA solve.
#pragma once

#include <cstdint>
#include <vector>

#include "dpslab.h"

namespace dps {

constexpr int kMaxSupport = 64;    // Gaussian support points per direction
constexpr int kMaxNz = 512;        // Chebyshev nodes
constexpr int kMaxFft = 4096;      // xy grid size per direction
constexpr int kMaxRadix = 64;      // largest prime factor of nx, ny
constexpr int kMaxStages = 24;

// Tensor-core z transforms (Nz <= 256, blocks of 128): canonical K-major, no-swizzle
// operand image of a rows x 128 bf16 operand, element (r, k) at
// r/8 * 2048 B + k/8 * 128 B + (r%8) * 16 B + (k%8) * 2 B (8 x 16-byte core
// matrices; K-direction stride 128 B, row-group stride 2048 B).
#ifdef __CUDACC__
#define DPS_HD __host__ __device__
#else
#define DPS_HD
#endif
constexpr int kZBlock = 128;       // row and K block of the z-transform GEMM
constexpr int kZMaxNz = 256;       // largest Nz on the tensor-core z transform (2 x 2 blocks)
DPS_HD inline constexpr int zimg_index(int r, int k) { return (r >> 3) * 1024 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7); }
// element offset of piece p of block (rb, kb) of an image with nb x nb
// blocks: each block is three contiguous zimg_index pieces of 128 x 128
DPS_HD inline constexpr size_t zimg_block(int rb, int kb, int nb, int p) {
    return (size_t(rb * nb + kb) * 3 + size_t(p)) * size_t(kZBlock) * kZBlock;
}

struct Complex {
    double re, im;
};

// Host-side tables of a plan (all double precision).
struct Tables {
    std::vector<double> zn;          // Chebyshev nodes z_j, descending, Sec. 5.2.2
    std::vector<double> wz;          // Clenshaw-Curtis weights times Hbar/2
    // Chebyshev transforms on the extrema grid split by the symmetry
    // cos(pi n (m-j)/m) = (-1)^n cos(pi n j/m), m = N-1: with
    // S_a = v_a + v_{m-a}, D_a = v_a - v_{m-a} (a < m-a; S = v at a middle
    // node), even coefficients use S and odd ones D:
    // cft[a][q], q < N: row q < (N+1)/2 is even n = 2q (input S_a), row
    // q >= (N+1)/2 is odd n = 2(q - (N+1)/2) + 1 (input D_a), a < (N+1)/2
    // (entries with no input are 0); stored input-major so that consecutive
    // output rows are consecutive in memory.
    std::vector<double> cft;
    // values at nodes a and m-a are E +/- O, E (O) the sum over even (odd) n:
    std::vector<double> tie;         // [n/2][a] = cos(pi n a/m), even n, a < (N+1)/2
    std::vector<double> tio;         // [(n-1)/2][a], odd n
    std::vector<double> j2l, j2d, j2u;   // diagonals (n-2, n, n+2) of J^2, Appendix A
    std::vector<double> u1, u2, v1, v2;  // 1^T J, 1^T J^2, (-1)^T J, (-1)^T J^2
    std::vector<double> t0, tH;      // T_n(s(0)), T_n(s(H))
    std::vector<double> wg;          // gauge weights int G_sigma(z) T_n(s(z)) dz
    std::vector<double> wgH;         // the same at z = H (wall-charge energy)
    std::vector<Complex> twx, twy;   // e^{-2 pi i k/n}
    std::vector<int> radx, rady;     // FFT radices (Stockham stages)
    // three bf16 pieces (x1 + x2 + x3) of the dense z transforms, 128 x 128
    // padded to whole 128 blocks, as zimg_index blocks (see zimg_block; empty when Nz > 256): coefficients from
    // node values (DCT-I form) and node values from coefficients
    std::vector<unsigned short> zimg_fwd, zimg_inv;
};

int derive(const dpslab_params& p, dpslab_derived& d);
int build_tables(const dpslab_params& p, const dpslab_derived& d, Tables& t);
bool fft_radices(int n, std::vector<int>& out);

}  // namespace dps
