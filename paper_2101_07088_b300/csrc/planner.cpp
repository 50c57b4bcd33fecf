// Host planner: parameter derivation (Sec. 5.1, Sec. 5.3, Table (ewconstraints))
// and the constant tables of a plan. No CUDA call in this file.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>

#include "internal.h"

namespace dps {
namespace {

constexpr double kPi = 3.14159265358979323846;

// d/dr of [erf(r/a1) - erf(r/a2)] / (4 pi r) (eps cancels in every ratio below);
// a2 = inf drops the second term (xi = 0).
double kernel_dr(double r, double a1, double a2) {
    auto term = [r](double a) {
        if (std::isinf(a)) return 0.0;
        const double x = r / a;
        return -std::erf(x) / (r * r) + 2.0 / (std::sqrt(kPi) * a) * std::exp(-x * x) / r;
    };
    return (term(a1) - term(a2)) / (4.0 * kPi);
}

double width2(double a1, double xi) {
    if (xi == 0.0) return INFINITY;
    if (std::isinf(xi)) return a1;
    return std::sqrt(a1 * a1 + 1.0 / (xi * xi));
}

// Smallest root of f on [lo, hi] where f goes from >= 0 to < 0: uniform scan,
// then bisection to the last bit.
double first_crossing(const std::function<double(double)>& f, double lo, double hi, int n) {
    double xp = lo, fp = f(lo);
    for (int i = 1; i <= n; ++i) {
        const double x = lo + (hi - lo) * double(i) / double(n);
        const double fx = f(x);
        if (fp >= 0.0 && fx < 0.0) {
            double a = xp, b = x;
            for (int it = 0; it < 200; ++it) {
                const double m = 0.5 * (a + b);
                if (m <= a || m >= b) break;
                if (f(m) >= 0.0) a = m; else b = m;
            }
            return b;
        }
        xp = x;
        fp = fx;
    }
    return NAN;
}

}  // namespace

bool fft_radices(int n, std::vector<int>& out) {
    out.clear();
    if (n < 1) return false;
    while (n % 4 == 0) { out.push_back(4); n /= 4; }
    while (n % 2 == 0) { out.push_back(2); n /= 2; }
    for (int p = 3; n > 1; p += 2) {
        while (n % p == 0) {
            if (p > kMaxRadix) return false;
            out.push_back(p);
            n /= p;
        }
        if (p > kMaxRadix && n > 1) return false;
    }
    return int(out.size()) <= kMaxStages;
}

int derive(const dpslab_params& p, dpslab_derived& d) {
    std::memset(&d, 0, sizeof(d));
    auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
    if (!pos(p.Lx) || !pos(p.Ly) || !pos(p.H) || !pos(p.gw) || !pos(p.eps)) return DPSLAB_ERR_INVALID_ARG;
    if (!(p.eps_b > 0.0) || !(p.eps_t > 0.0)) return DPSLAB_ERR_INVALID_ARG;   // may be +inf
    if (p.nx < 4 || p.ny < 4 || p.nx > kMaxFft || p.ny > kMaxFft) return DPSLAB_ERR_GRID;
    if (p.nz != 0 && (p.nz < 4 || p.nz > kMaxNz)) return DPSLAB_ERR_GRID;
    if (p.precision != DPSLAB_FP64 && p.precision != DPSLAB_MIXED && p.precision != DPSLAB_MIXED_SIMT)
        return DPSLAB_ERR_UNSUPPORTED;
    if (!(p.xi >= 0.0) || !(p.r_cut >= 0.0) || !(p.n_sigma >= 0.0)) return DPSLAB_ERR_INVALID_ARG;

    // Table (ewconstraints)
    double c_h, n_g;
    if (std::fabs(p.tol - 1e-4) < 1e-12) { c_h = 1.4; n_g = 12.0; }
    else if (std::fabs(p.tol - 5e-4) < 1e-12) { c_h = 1.2; n_g = 10.0; }
    else return DPSLAB_ERR_INVALID_ARG;
    const double n_sigma = p.n_sigma > 0.0 ? p.n_sigma : n_g / (2.0 * c_h);

    d.nx = p.nx;
    d.ny = p.ny;
    d.hx = p.Lx / p.nx;
    d.hy = p.Ly / p.ny;
    d.h = std::max(d.hx, d.hy);

    double xi = p.xi;
    if (xi == 0.0) {
        if (p.r_cut > 0.0) {
            // the grid resolves g_w: xi from the averaged-kernel cutoff rule
            const double a1 = 2.0 * p.gw;
            const double ref = kernel_dr(p.r_cut, a1, INFINITY);
            auto f = [&](double x) { return std::fabs(kernel_dr(p.r_cut, a1, width2(a1, x)) / ref) - p.tol; };
            xi = first_crossing(f, 0.05 / p.gw, 400.0 / p.gw, 8000);
        } else {
            const double gt_rule = c_h * d.h;            // Sec. 5.1
            if (!(gt_rule > p.gw)) return DPSLAB_ERR_INVALID_ARG;
            xi = 1.0 / (2.0 * std::sqrt(gt_rule * gt_rule - p.gw * p.gw));   // Eq. (gt)
        }
        if (!std::isfinite(xi)) return DPSLAB_ERR_INVALID_ARG;
    }
    d.xi = xi;
    d.gt = std::isinf(xi) ? p.gw : std::sqrt(1.0 / (4.0 * xi * xi) + p.gw * p.gw);   // Eq. (gt)
    d.n_sigma = n_sigma;
    d.HE = n_sigma * d.gt;                                                    // Eq. (He)

    d.r_nf = 0.0;
    d.r_cut = p.r_cut;
    if (std::isinf(xi)) {
        d.r_cut = 0.0;                      // no splitting: no near field
    } else if (d.r_cut == 0.0) {
        const double a1 = std::sqrt(2.0) * p.gw;                              // Eq. (rnf), pointwise kernel
        const double a2 = width2(a1, xi);
        auto f = [&](double r) { return std::fabs(kernel_dr(r, a1, a2) / kernel_dr(r, a1, INFINITY)) - p.tol; };
        d.r_nf = first_crossing(f, 1e-6 / xi, 40.0 / xi, 4000);
        if (!std::isfinite(d.r_nf)) return DPSLAB_ERR_INVALID_ARG;
        d.r_cut = d.r_nf + n_sigma * p.gw;
    }

    d.nz = p.nz != 0 ? p.nz : int(std::ceil(kPi * (p.H + 6.0 * d.HE) / (2.0 * d.h)));   // Sec. 5.1
    if (d.nz < 4 || d.nz > kMaxNz) return DPSLAB_ERR_GRID;
    d.a = -3.0 * d.HE;
    d.b = p.H + 3.0 * d.HE;
    d.Hbar = d.b - d.a;
    d.kmax = kPi / d.h;

    d.support_x = int(std::floor(2.0 * d.HE / d.hx)) + 1;
    d.support_y = int(std::floor(2.0 * d.HE / d.hy)) + 1;
    if (d.support_x > p.nx || d.support_y > p.ny) return DPSLAB_ERR_GRID;
    if (d.support_x + 1 > kMaxSupport || d.support_y + 1 > kMaxSupport) return DPSLAB_ERR_GRID;
    std::vector<int> r;
    if (!fft_radices(p.nx, r) || !fft_radices(p.ny, r)) return DPSLAB_ERR_GRID;

    if (d.r_cut > 0.0 && d.r_cut >= 0.5 * std::min(p.Lx, p.Ly)) return DPSLAB_ERR_CUTOFF_TOO_LARGE;
    d.violations = 0;
    if (2.0 * d.HE >= p.H) d.violations |= DPSLAB_VIOL_FAR_FIELD;
    if (d.r_cut >= p.H) d.violations |= DPSLAB_VIOL_NEAR_FIELD;
    if (p.strict && d.violations) return DPSLAB_ERR_SPLIT_CONSTRAINT;
    return DPSLAB_OK;
}

int build_tables(const dpslab_params& p, const dpslab_derived& d, Tables& t) {
    const int N = d.nz;
    const int m = N - 1;
    // cos(pi k / m), k = 0 .. 2m-1, in extended precision
    std::vector<double> cs(2 * m);
    for (int k = 0; k < 2 * m; ++k) cs[k] = double(cosl(3.141592653589793238462643383279503L * k / m));

    t.zn.resize(N);
    for (int j = 0; j < N; ++j) t.zn[j] = d.a + 0.5 * d.Hbar * (1.0 + cs[j]);

    // Clenshaw-Curtis weights on [-1, 1] (closed form), scaled by Hbar/2
    t.wz.assign(N, 0.0);
    for (int j = 0; j < N; ++j) {
        long double s = 1.0L;
        for (int k = 1; 2 * k <= m; ++k) {
            const long double bk = (2 * k == m) ? 1.0L : 2.0L;
            s -= bk / (4.0L * k * k - 1.0L) * cs[(size_t(2 * k) * j) % (2 * m)];   // cos(2 pi k j / m)
        }
        const long double cj = (j == 0 || j == m) ? 1.0L : 2.0L;
        t.wz[j] = double(cj / m * s * 0.5L * d.Hbar);
    }

    // Chebyshev transforms on the extrema grid (DCT-I form):
    // fhat_n = (2/m) w_n sum_j w_j v_j cos(pi n j/m), w = 1/2 at the ends
    const int JE = (N + 1) / 2, JO = N / 2;
    auto fwd = [&](int n, int j) {
        const double wj = (j == 0 || j == m) ? 0.5 : 1.0;
        const double wn = (n == 0 || n == m) ? 0.5 : 1.0;
        return 2.0 / m * wj * wn * cs[(size_t(n) * j) % (2 * m)];
    };
    t.cft.assign(size_t(JE) * N, 0.0);
    t.tie.assign(size_t(JE) * JE, 0.0);
    t.tio.assign(size_t(JO) * JE, 0.0);
    for (int a = 0; a < JE; ++a) {
        for (int q = 0; q < JE; ++q) t.cft[size_t(a) * N + q] = fwd(2 * q, a);
        if (a < JO)
            for (int q = 0; q < JO; ++q) t.cft[size_t(a) * N + JE + q] = fwd(2 * q + 1, a);
        for (int r = 0; r < JE; ++r) t.tie[size_t(r) * JE + a] = cs[(size_t(2 * r) * a) % (2 * m)];
        for (int r = 0; r < JO; ++r) t.tio[size_t(r) * JE + a] = cs[(size_t(2 * r + 1) * a) % (2 * m)];
    }

    // dense transforms for the tensor-core path: each entry x as three bf16
    // pieces x1 + x2 + x3 (round to nearest even at each step)
    if (N <= kZMaxNz) {
        auto bf16 = [](double x) -> unsigned short {
            const float f = float(x);
            uint32_t u;
            std::memcpy(&u, &f, 4);
            u += 0x7FFFu + ((u >> 16) & 1u);
            return static_cast<unsigned short>(u >> 16);
        };
        auto bf16v = [](unsigned short h) -> double {
            const uint32_t u = uint32_t(h) << 16;
            float f;
            std::memcpy(&f, &u, 4);
            return double(f);
        };
        // piece 1 on a fixed-point grid: rint(x 128/s) s/128 with s the power
        // of two at or above the row's largest |entry| (an integer of at most
        // 8 bits times a power of two, exact in bf16); pieces 2 and 3 the bf16
        // roundings of what remains
        auto image = [&](std::vector<unsigned short>& img, const std::function<double(int, int)>& A) {
            const int nb = (N + kZBlock - 1) / kZBlock, R = nb * kZBlock;
            img.assign(size_t(nb) * nb * 3 * kZBlock * kZBlock, 0);
            for (int r = 0; r < R; ++r) {
                double amax = 0.0;
                for (int k = 0; k < R; ++k) amax = std::max(amax, std::fabs(A(r, k)));
                int e = 0;
                if (amax > 0.0) std::frexp(amax, &e);
                const double sc = std::ldexp(1.0, e);     // > amax
                for (int k = 0; k < R; ++k) {
                    double x = A(r, k);
                    const double p1 = std::rint(x * 128.0 / sc) * (sc / 128.0);
                    const int rb = r / kZBlock, kb = k / kZBlock, ri = r % kZBlock, ki = k % kZBlock;
                    img[zimg_block(rb, kb, nb, 0) + zimg_index(ri, ki)] = bf16(p1);
                    x -= p1;
                    for (int piece = 1; piece < 3; ++piece) {
                        const unsigned short h = bf16(x);
                        img[zimg_block(rb, kb, nb, piece) + zimg_index(ri, ki)] = h;
                        x -= bf16v(h);
                    }
                }
            }
        };
        image(t.zimg_fwd, [&](int n, int j) { return (n < N && j < N) ? fwd(n, j) : 0.0; });
        image(t.zimg_inv, [&](int j, int n) { return (n < N && j < N) ? cs[(size_t(n) * j) % (2 * m)] : 0.0; });
    }

    // Appendix A: J maps coefficients of a function to those of its integral
    // (constant excluded): J[1][0] = 1, J[1][2] = -1/2, J[n][n-1] = 1/(2n),
    // J[n][n+1] = -1/(2n), dropping indices >= N.
    auto J = [N](int n, int k) -> double {
        if (n <= 0 || n >= N || k < 0 || k >= N) return 0.0;
        if (n == 1) return k == 0 ? 1.0 : (k == 2 ? -0.5 : 0.0);
        if (k == n - 1) return 1.0 / (2.0 * n);
        if (k == n + 1) return -1.0 / (2.0 * n);
        return 0.0;
    };
    auto J2 = [&](int n, int k) -> double {
        double s = 0.0;
        for (int q = n - 1; q <= n + 1; q += 2) s += J(n, q) * J(q, k);   // row n of J is nonzero at n -/+ 1 only
        return s;
    };
    t.j2l.assign(N, 0.0);
    t.j2d.assign(N, 0.0);
    t.j2u.assign(N, 0.0);
    t.u1.assign(N, 0.0);
    t.u2.assign(N, 0.0);
    t.v1.assign(N, 0.0);
    t.v2.assign(N, 0.0);
    for (int n = 0; n < N; ++n) {
        t.j2l[n] = J2(n, n - 2);
        t.j2d[n] = J2(n, n);
        t.j2u[n] = J2(n, n + 2);
    }
    for (int k = 0; k < N; ++k) {
        double a = 0, b = 0, c = 0, e = 0;
        for (int n = std::max(0, k - 2); n <= std::min(N - 1, k + 2); ++n) {
            const double sg = (n % 2 == 0) ? 1.0 : -1.0;
            a += J(n, k);
            b += J2(n, k);
            c += sg * J(n, k);
            e += sg * J2(n, k);
        }
        t.u1[k] = a;
        t.u2[k] = b;
        t.v1[k] = c;
        t.v2[k] = e;
    }

    // T_n at z = 0 and z = H
    auto cheb_row = [N](long double s, std::vector<double>& out) {
        out.assign(N, 0.0);
        long double tm = 1.0L, tc = s;
        out[0] = 1.0;
        if (N > 1) out[1] = double(s);
        for (int n = 2; n < N; ++n) {
            const long double tn = 2.0L * s * tc - tm;
            out[n] = double(tn);
            tm = tc;
            tc = tn;
        }
    };
    const long double s0 = 2.0L * (0.0L - d.a) / d.Hbar - 1.0L;
    const long double sH = 2.0L * ((long double)p.H - d.a) / d.Hbar - 1.0L;
    cheb_row(s0, t.t0);
    cheb_row(sH, t.tH);

    // gauge weights: int G_sigma(z) T_n(sc + 2 z/Hbar) dz, sigma = 1/(2 xi),
    // by the trapezoid rule on [-14 sigma, 14 sigma] (spectrally accurate for a
    // Gaussian times a polynomial): the z part of the gamma^{1/2} average of a
    // Chebyshev series at the height whose scaled coordinate is sc (z = 0 for
    // the gauge; z = 0 and z = H for the wall-charge energy)
    auto gauge_row = [&](long double sc, const std::vector<double>& plain, std::vector<double>& out) {
        if (std::isinf(d.xi)) {
            out = plain;
            return;
        }
        const long double sig = 0.5L / d.xi;
        const int M = 601;   // step 0.047 sigma: the aliasing error exp(-2 pi^2 sigma^2 / dz^2) is far below 1e-16
        const long double zlo = -14.0L * sig, dzs = 28.0L * sig / (M - 1);
        std::vector<long double> acc(N, 0.0L);
        for (int i = 0; i < M; ++i) {
            const long double z = zlo + dzs * i;
            const long double g = expl(-z * z / (2.0L * sig * sig)) /
                                  (sig * sqrtl(2.0L * 3.141592653589793238462643383279503L));
            const long double w = (i == 0 || i == M - 1) ? 0.5L : 1.0L;
            long double tm = 1.0L, s = sc + 2.0L * z / d.Hbar, tc = s;
            acc[0] += w * g;
            if (N > 1) acc[1] += w * g * s;
            for (int n = 2; n < N; ++n) {
                const long double tn = 2.0L * s * tc - tm;
                acc[n] += w * g * tn;
                tm = tc;
                tc = tn;
            }
        }
        out.resize(N);
        for (int n = 0; n < N; ++n) out[n] = double(acc[n] * dzs);
    };
    gauge_row(s0, t.t0, t.wg);
    gauge_row(sH, t.tH, t.wgH);

    // FFT twiddles and radices
    auto tw = [](int n, std::vector<Complex>& out) {
        out.resize(n);
        for (int k = 0; k < n; ++k) {
            const long double a = -2.0L * 3.141592653589793238462643383279503L * k / n;
            out[k] = Complex{double(cosl(a)), double(sinl(a))};
        }
    };
    tw(p.nx, t.twx);
    tw(p.ny, t.twy);
    if (!fft_radices(p.nx, t.radx) || !fft_radices(p.ny, t.rady)) return DPSLAB_ERR_GRID;
    return DPSLAB_OK;
}

}  // namespace dps
