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
// Radices 2 and 4 have dedicated butterflies; any other radix uses the
// direct R-point sum with table twiddles.
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

}  // namespace dps
