// Block-cooperative mixed-radix Stockham FFT in shared memory.
//
// B sequences of length n are stored back to back (sequence b at offset
// b * n) in buffer `a`; `b` is a scratch buffer of the same size. Stage s
// with radix R (Ns = product of the previous radices) reads a[j + r n/R],
// multiplies by the twiddle w^(r (j mod Ns) n/(Ns R)), takes an R-point DFT
// and writes b[(j div Ns) Ns R + (j mod Ns) + r' Ns]: the self-sorting
// (autosort) form, so the result is in natural order with no bit reversal.
// `tw` holds w^k = e^{-2 pi i k/n}, k < n; dir = -1 is the forward
// transform sum_x f(x) e^{-2 pi i k x/n}, dir = +1 the unnormalised inverse.
// Radices 2 and 4 have dedicated butterflies, 3, 5 and 7 a paired one
// (odd_butterfly); any other radix uses the direct R-point sum with table
// twiddles.
#pragma once

#include <cuda_runtime.h>

namespace dps {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// multiply by -i (dir = -1) or +i (dir = +1)
__device__ __forceinline__ double2 cmul_i(double2 a, int dir) {
    return dir < 0 ? make_double2(a.y, -a.x) : make_double2(-a.y, a.x);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul_i(float2 a, int dir) {
    return dir < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <class C>
__device__ __forceinline__ C twiddle(const C* tw, int k, int dir) {
    const C w = tw[k];
    return dir < 0 ? w : cconj(w);
}

// Odd radix R = 3, 5, 7: the inputs get their stage twiddle once, then the
// R-point DFT pairs inputs r and R - r: with S = v_r + v_{R-r},
// D = v_r - v_{R-r}, output r' gains S cos(2 pi k/R) + i dir D sin(2 pi k/R),
// k = r r' mod R, the constants read from the twiddle table
// (tw[k n/R] = e^{-2 pi i k/R}).
template <int R, class C>
__device__ __forceinline__ void odd_butterfly(const C* x, C* y, int j, int nR, int out0, int Ns, int jm, int step,
                                              const C* tw, int dir) {
    constexpr int h = (R - 1) / 2;
    C v[R];
    v[0] = x[j];
#pragma unroll
    for (int r = 1; r < R; ++r) {
        v[r] = x[j + r * nR];
        if (jm) v[r] = cmul(v[r], twiddle(tw, r * jm * step, dir));
    }
    C S[h], D[h];
    C y0 = v[0];
#pragma unroll
    for (int m = 1; m <= h; ++m) {
        S[m - 1] = cadd(v[m], v[R - m]);
        D[m - 1] = csub(v[m], v[R - m]);
        y0 = cadd(y0, S[m - 1]);
    }
    y[out0] = y0;
    C cs[R];
#pragma unroll
    for (int k = 1; k < R; ++k) cs[k] = tw[k * nR];
    const auto sd = decltype(v[0].x)(dir);
#pragma unroll
    for (int rp = 1; rp < R; ++rp) {
        auto re = v[0].x, im = v[0].y;
#pragma unroll
        for (int m = 1; m <= h; ++m) {
            const int k = (m * rp) % R;
            const auto c = cs[k].x, sn = -cs[k].y * sd;   // cos(2 pi k/R), dir sin(2 pi k/R)
            re += S[m - 1].x * c - sn * D[m - 1].y;
            im += S[m - 1].y * c + sn * D[m - 1].x;
        }
        C o;
        o.x = re;
        o.y = im;
        y[out0 + rp * Ns] = o;
    }
}

// Returns the buffer holding the result (a or b). Ends with __syncthreads().
template <class C>
__device__ inline C* block_fft(C* a, C* b, const C* tw, int n, int nseq, const int* radices, int nstages, int dir) {
    int Ns = 1;
    for (int s = 0; s < nstages; ++s) {
        const int R = radices[s];
        const int nR = n / R;
        const int step = n / (Ns * R);
        const int total = nseq * nR;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int q = t / nR;
            const int j = t - q * nR;
            const C* x = a + q * n;
            C* y = b + q * n;
            const int jm = j % Ns;
            const int out0 = (j / Ns) * Ns * R + jm;
            if (R == 4) {
                C v0 = x[j];
                C v1 = x[j + nR];
                C v2 = x[j + 2 * nR];
                C v3 = x[j + 3 * nR];
                if (jm) {
                    v1 = cmul(v1, twiddle(tw, jm * step, dir));
                    v2 = cmul(v2, twiddle(tw, 2 * jm * step, dir));
                    v3 = cmul(v3, twiddle(tw, 3 * jm * step, dir));
                }
                const C s02 = cadd(v0, v2), d02 = csub(v0, v2);
                const C s13 = cadd(v1, v3), d13 = cmul_i(csub(v1, v3), dir);
                y[out0] = cadd(s02, s13);
                y[out0 + Ns] = cadd(d02, d13);
                y[out0 + 2 * Ns] = csub(s02, s13);
                y[out0 + 3 * Ns] = csub(d02, d13);
            } else if (R == 2) {
                C v0 = x[j];
                C v1 = x[j + nR];
                if (jm) v1 = cmul(v1, twiddle(tw, jm * step, dir));
                y[out0] = cadd(v0, v1);
                y[out0 + Ns] = csub(v0, v1);
            } else if (R == 3) {
                odd_butterfly<3>(x, y, j, nR, out0, Ns, jm, step, tw, dir);
            } else if (R == 5) {
                odd_butterfly<5>(x, y, j, nR, out0, Ns, jm, step, tw, dir);
            } else if (R == 7) {
                odd_butterfly<7>(x, y, j, nR, out0, Ns, jm, step, tw, dir);
            } else {
                // y[out0 + r' Ns] = sum_r x[j + r nR] w^(r (jm step + r' nR))
                for (int rp = 0; rp < R; ++rp) {
                    const int e = (jm * step + rp * nR) % n;
                    C acc = x[j];
                    int idx = 0;
                    for (int r = 1; r < R; ++r) {
                        idx += e;
                        if (idx >= n) idx -= n;
                        acc = cadd(acc, cmul(x[j + r * nR], twiddle(tw, idx, dir)));
                    }
                    y[out0 + rp * Ns] = acc;
                }
            }
        }
        __syncthreads();
        C* tmp = a;
        a = b;
        b = tmp;
        Ns *= R;
    }
    return a;
}


// ---------------------------------------------------------------------------
// Power-of-two sizes 32 <= n <= 4096: register radix-16 Stockham passes.
//
// Each thread owns one slot j < n/16 of one sequence q and keeps 16 values
// in registers. Pass 1 (radix 16, Ns = 1) reads x[j + r n/16] through the
// caller's load functor; middle passes (radix 16, Ns = 16^p) exchange through
// one padded shared buffer; the last pass (radix RL = n/16^a in {2,4,8,16},
// 16/RL butterflies per thread) hands x[j + g n/16] to the store functor, in
// natural order. Stage s with radix R and Ns multiplies input r of butterfly
// j by w^(r (j mod Ns) n/(Ns R)), takes the R-point DFT and writes output r'
// to (j - j mod Ns) R + j mod Ns + r' Ns (the autosort form of the generic
// routine above). The R-point DFTs are fixed Cooley-Tukey splits (16 = 4x4,
// 8 = 2x4) with the constants cos/sin(pi m/8) written out.
// ---------------------------------------------------------------------------

// one spare slot every 16 elements: conflict-free strided exchanges
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

template <class C> struct CScalar;
template <> struct CScalar<float2> { using T = float; };
template <> struct CScalar<double2> { using T = double; };

template <class C>
__device__ __forceinline__ C cmake(double x, double y) {
    C c;
    c.x = typename CScalar<C>::T(x);
    c.y = typename CScalar<C>::T(y);
    return c;
}

// v[0], v[S] <- 2-point DFT
template <int S, class C>
__device__ __forceinline__ void dft2(C* v) {
    const C a = v[0], b = v[S];
    v[0] = cadd(a, b);
    v[S] = csub(a, b);
}

// v[0], v[S], v[2S], v[3S] <- 4-point DFT with kernel e^{dir 2 pi i nk/4}
template <int S, class C>
__device__ __forceinline__ void dft4(C* v, int dir) {
    const C a = v[0], b = v[S], c = v[2 * S], d = v[3 * S];
    const C s02 = cadd(a, c), d02 = csub(a, c), s13 = cadd(b, d), d13 = cmul_i(csub(b, d), dir);
    v[0] = cadd(s02, s13);
    v[S] = cadd(d02, d13);
    v[2 * S] = csub(s02, s13);
    v[3 * S] = csub(d02, d13);
}

// cos and sin of 2 pi m/16
__device__ __forceinline__ constexpr double cos16(int m) {
    constexpr double c8 = 0.92387953251128675613, s8 = 0.38268343236508977173, r2 = 0.70710678118654752440;
    const double t[16] = {1.0, c8, r2, s8, 0.0, -s8, -r2, -c8, -1.0, -c8, -r2, -s8, 0.0, s8, r2, c8};
    return t[m & 15];
}
__device__ __forceinline__ constexpr double sin16(int m) { return cos16(m - 4); }

// multiply by e^{dir 2 pi i m/16} (m known at compile time after unrolling)
template <class C>
__device__ __forceinline__ C rot16(C a, int m, int dir) {
    m &= 15;
    if (m == 0) return a;
    if (m == 4) return cmul_i(a, dir);
    if (m == 8) return cmake<C>(-a.x, -a.y);
    if (m == 12) return cmul_i(a, -dir);
    return cmul(a, cmake<C>(cos16(m), dir * sin16(m)));
}

// v[0], v[S], ..., v[7S] <- 8-point DFT: two 4-point DFTs of the even and
// odd inputs, combined with e^{dir 2 pi i k/8}
template <int S, class C>
__device__ __forceinline__ void dft8(C* v, int dir) {
    C e[4] = {v[0], v[2 * S], v[4 * S], v[6 * S]};
    C o[4] = {v[S], v[3 * S], v[5 * S], v[7 * S]};
    dft4<1>(e, dir);
    dft4<1>(o, dir);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const C t = rot16(o[k], 2 * k, dir);
        v[k * S] = cadd(e[k], t);
        v[(k + 4) * S] = csub(e[k], t);
    }
}

// v[0..15] <- 16-point DFT: 4-point DFTs over n1 for each n2 (input
// n = 4 n1 + n2), twiddles e^{dir 2 pi i n2 k1/16}, 4-point DFTs over n2,
// output k = k1 + 4 k2
template <class C>
__device__ __forceinline__ void dft16(C* v, int dir) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<4>(v + n2, dir);
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) v[n2 + 4 * k1] = rot16(v[n2 + 4 * k1], n2 * k1, dir);
    C t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C* y = v + 4 * k1;
        dft4<1>(y, dir);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = y[k2];
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = t[k];
}

template <int R, int S, class C>
__device__ __forceinline__ void dft_r(C* v, int dir) {
    if constexpr (R == 2) dft2<S>(v);
    else if constexpr (R == 4) dft4<S>(v, dir);
    else if constexpr (R == 8) dft8<S>(v, dir);
    else dft16(v, dir);
}

// v[S r] *= w^(r e), r = 1..R-1, w = e^{dir 2 pi i/n}, from the table
// tw[k] = e^{-2 pi i k/n} (r e < n)
template <int R, int S, class C>
__device__ __forceinline__ void twiddle_r(C* v, const C* tw, int e, int dir) {
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const C w = tw[r * e];
        v[S * r] = cmul(v[S * r], dir < 0 ? w : cconj(w));
    }
}

template <int RL, class C>
__device__ __forceinline__ void last_pass(C* v, const C* tw, int j, int n16, int dir) {
    constexpr int S = 16 / RL;
#pragma unroll
    for (int m = 0; m < S; ++m) {
        twiddle_r<RL, S>(v + m, tw, j + m * n16, dir);
        dft_r<RL, S>(v + m, dir);
    }
}

// FFT of nseq sequences of length n = 2^logn (32 <= n <= 4096) with
// nseq * n/16 <= blockDim.x threads; thread s < nseq n/16 takes slot
// (q, j) = (s mod nseq, s div nseq) when QF (neighbouring threads on
// neighbouring sequences: column transforms) and (s div (n/16), s mod (n/16))
// otherwise (row transforms). buf: nseq * n * 17/16 elements of shared
// memory. load(q, i) returns input i of sequence q; store(q, i, v) receives
// output i, after a barrier (it may write buf). All threads of the block
// must call this function; it ends with the stores done by each thread.
// kSyncLoad: a barrier between the first pass's loads and its writes, for
// loads that read staged input from buf itself. tw: the twiddle table (n
// entries). Row transforms read the global table where it is (it stays in
// L1). Column transforms pass tw_fill = tw in shared memory and tw_src, the
// global table: it is copied here while the first pass's loads are in
// flight (that pass needs no twiddles, and the barrier after its writes
// precedes the first use).
// kPaired (row transforms, nseq even): the sequences come in pairs
// (2 m, 2 m + 1) on neighbouring lanes, thread s taking
// (q, j) = (2 (s div 2 n16) + s mod 2, (s div 2) mod n16), with sequences
// n + n16 + 8 elements apart so that the two lanes of a pair use opposite
// halves of the banks; the outputs stay in registers: store(q, j, act, v)
// receives all 16 of a thread (output j + g n16 in v[g]), with no barrier
// before it, and every thread calls it, so that it may exchange values
// between the two lanes of a pair.
template <bool QF, bool kSyncLoad = false, bool kPaired = false, class C, class Load, class Store>
__device__ __forceinline__ void fft_pow2(C* buf, const C* tw, int n, int logn, int nseq, int dir, Load load,
                                         Store store, C* tw_fill = nullptr, const C* tw_src = nullptr) {
    const int l16 = logn - 4, n16 = 1 << l16;
    const int s = threadIdx.x;
    const bool act = s < (nseq << l16);
    const int q = QF ? s % nseq : kPaired ? 2 * (s >> (l16 + 1)) + (s & 1) : s >> l16;
    const int j = QF ? s / nseq : kPaired ? (s >> 1) & (n16 - 1) : s & (n16 - 1);
    const int sstr = n + n16 + (kPaired ? 8 : 0);
    auto at = [&](int i) { return QF ? pad16(i * nseq + q) : q * sstr + pad16(i); };
    const int a = (logn - 1) >> 2;            // radix-16 passes
    const int lrl = logn - 4 * a;             // log2 of the last radix
    C v[16];
    if (act) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = load(q, j + r * n16);
    }
    if (tw_fill)
        for (int i = threadIdx.x; i < n; i += blockDim.x) tw_fill[i] = tw_src[i];
    if constexpr (kSyncLoad) __syncthreads();
    if (act) {
        dft16(v, dir);
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[at(16 * j + r)] = v[r];
    }
    __syncthreads();
    int lNs = 4;
    for (int p = 1; p < a; ++p, lNs += 4) {
        const int jm = j & ((1 << lNs) - 1);
        if (act) {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = buf[at(j + r * n16)];
            twiddle_r<16, 1>(v, tw, jm << (logn - 4 - lNs), dir);
            dft16(v, dir);
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int r = 0; r < 16; ++r) buf[at(((j - jm) << 4) + jm + (r << lNs))] = v[r];
        }
        __syncthreads();
    }
    if (act) {
#pragma unroll
        for (int g = 0; g < 16; ++g) v[g] = buf[at(j + g * n16)];
        if (lrl == 1) last_pass<2>(v, tw, j, n16, dir);
        else if (lrl == 2) last_pass<4>(v, tw, j, n16, dir);
        else if (lrl == 3) last_pass<8>(v, tw, j, n16, dir);
        else last_pass<16>(v, tw, j, n16, dir);
    }
    if constexpr (kPaired) {
        store(q, j, act, v);
    } else {
        __syncthreads();
        if (act) {
#pragma unroll
            for (int g = 0; g < 16; ++g) store(q, j + g * n16, v[g]);
        }
    }
}

}  // namespace dps
