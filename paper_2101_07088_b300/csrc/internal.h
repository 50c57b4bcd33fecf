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

struct Complex {
    double re, im;
};

// Host-side tables of a plan (all double precision).
struct Tables {
    std::vector<double> zn;          // Chebyshev nodes z_j, descending, Sec. 5.2.2
    std::vector<double> wz;          // Clenshaw-Curtis weights times Hbar/2
    std::vector<double> cf;          // [n][j]: node values -> Chebyshev coefficients
    std::vector<double> ti;          // [j][n]: T_n(s_j) = cos(pi n j/(N-1))
    std::vector<double> j2l, j2d, j2u;   // diagonals (n-2, n, n+2) of J^2, Appendix A
    std::vector<double> u1, u2, v1, v2;  // 1^T J, 1^T J^2, (-1)^T J, (-1)^T J^2
    std::vector<double> t0, tH;      // T_n(s(0)), T_n(s(H))
    std::vector<double> wg;          // gauge weights int G_sigma(z) T_n(s(z)) dz
    std::vector<Complex> twx, twy;   // e^{-2 pi i k/n}
    std::vector<int> radx, rady;     // FFT radices (Stockham stages)
};

int derive(const dpslab_params& p, dpslab_derived& d);
int build_tables(const dpslab_params& p, const dpslab_derived& d, Tables& t);
bool fft_radices(int n, std::vector<int>& out);

}  // namespace dps
