// fl_common.cuh -- device helpers shared by the kernels of libfl.so:
// complex arithmetic, sincospi by precision, the per-band descriptor, and the
// shared-memory Stockham FFT used by every NFFT (Kunis & Melzer, Section 4:
// each band's Fourier factor A~ is one NFFT, i.e. deconvolution, one FFT of
// the oversampled grid, and window interpolation).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fl {

// Float pairs (the FP64-accuracy form FL_FP64_FF): a value hi + lo, about 48
// significant bits from FP32 arithmetic alone (double-length arithmetic after
// Dekker, 1971: Knuth's error-free sum and the FMA error-free product).  The
// pairs are kept unnormalised: a sum or product returns the exact rounded
// leading part and the collected low-order terms without the final fast
// two-sum, so |lo| may grow to a few ulp(hi), or exceed |hi| after
// cancellation.  The value is always hi + lo, and the error of each operation
// stays a few 2^-48 of the operands' magnitudes (|a| + |b|, |a| |b|), the
// norm-wise bound an FFT needs.  Values enter as pairs rounded from FP64 and
// leave through double(hi) + double(lo).
struct __align__(8) ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr ff(float v) : hi(v), lo(0.f) {}
    // exact for |v| <= 2^24 (the integers used here are transform indices)
    __host__ __device__ constexpr ff(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ constexpr ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ explicit constexpr operator double() const { return (double)hi + (double)lo; }
};
struct __align__(16) ffc {
    ff x, y;
};

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator+(ff a, ff b) {
    const float s = a.hi + b.hi;                      // Knuth: s + err == a.hi + b.hi
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b.hi - bb);
    return ff(s, err + (a.lo + b.lo));
}
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);             // the rounding error of p, exactly
    return ff(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
// s * a for s = +-1 or a power of two (the sign factors of the butterflies):
// exact
__device__ __forceinline__ ff operator*(int s, ff a) { return ff((float)s * a.hi, (float)s * a.lo); }
// through double: used only for set-up values (1 / power of two)
__device__ __forceinline__ ff operator/(ff a, ff b) { return ff((double)a / (double)b); }
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }

template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<ff> { using type = ffc; };
template <typename T> using C_t = typename cplx<T>::type;

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return {a.x * s, a.y * s}; }
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }
// float pairs: through double sincospi, rounded to a pair (relative error ~2^-48)
__device__ __forceinline__ void sincospi_t(ff x, ff* s, ff* c) {
    double sd, cd;
    sincospi((double)x, &sd, &cd);
    *s = ff(sd);
    *c = ff(cd);
}

// exp(i * pi * x)
template <typename T> __device__ __forceinline__ C_t<T> expipi(T x) {
    T s, c;
    sincospi_t(x, &s, &c);
    return {c, s};
}

// k x mod 1 in [-1/2, 1/2) (turns).  The product is split exactly by one FMA
// (k x = p + e, Dekker's two-product), so the reduced phase is correct to
// about 2^-53 however large k x is; a rounded k x alone would lose
// ulp(k x) / 2, 2^-31 turns at k x = 2^22.
__device__ __forceinline__ double frac_turns(double k, double x) {
    const double p = k * x;
    const double e = fma(k, x, -p);
    double f = (p - rint(p)) + e;
    if (f >= 0.5) f -= 1.0;
    if (f < -0.5) f += 1.0;
    return f;
}

// Stage twiddle tables.  In a length-L transform whose first stage has radix
// 2^FIRST, every later stage (radix R, span NS = 2^d) multiplies input r of job
// jj by w^(r k), w = exp(SIGN 2 pi i / (NS R)), k = jj mod NS.  Those values are
// tabulated at plan time (FP64, rounded once) for SIGN = +1 in pairs
// (r, r + 1) = (2p + 1, 2p + 2):
//   tab[tw_region(LOG2L, FIRST) + tw_off(LOG2L, FIRST, d) + 2 NS p + 2 k + (r - 1) % 2],
// so a job reads its R - 1 factors as R/2 adjacent pairs (one 16-byte load
// each in float; consecutive jobs, consecutive pairs) and SIGN = -1 takes the
// conjugate.  The pair slot of r = R (beyond the last factor) holds zero.
constexpr int kTwMinLog = 6, kTwMaxLog = 12;
constexpr int kTwRegion = 2 << kTwMaxLog;                   // entries per (LOG2L, FIRST)
constexpr int kTwEntries = (kTwMaxLog - kTwMinLog + 1) * 2 * kTwRegion;

__host__ __device__ constexpr int tw_last_log(int LOG2L, int FIRST) {
    return (LOG2L - FIRST) - 4 * (((LOG2L - FIRST) + 3) / 4 - 1);
}
// log2 of the radix of the stage of span 2^d (d = FIRST, FIRST + 4, ...)
__host__ __device__ constexpr int tw_stage_log(int LOG2L, int FIRST, int d) {
    return d == LOG2L - tw_last_log(LOG2L, FIRST) ? tw_last_log(LOG2L, FIRST) : 4;
}
__host__ __device__ constexpr int tw_off(int LOG2L, int FIRST, int d) {
    int off = 0;
    for (int e = FIRST; e < d; e += 4) off += (1 << tw_stage_log(LOG2L, FIRST, e)) << e;
    return off;
}
__host__ __device__ constexpr int tw_region(int LOG2L, int FIRST) {
    return ((LOG2L - kTwMinLog) * 2 + (FIRST - 3)) * kTwRegion;
}

// Kaiser-Bessel window in grid units, phi(t) = sinh(b sqrt(m^2 - t^2)) / sqrt(m^2 - t^2),
// |t| <= m (limit b at |t| = m).
template <typename T> __device__ __forceinline__ T kb_window(T t, T m, T b) {
    const T s2 = m * m - t * t;
    if (!(s2 > (T)0)) return b;
    const T r = sqrt(s2);
    return sinh(b * r) / r;
}

// Per-band descriptor (bands 1..levels; band 0 is Z^0).  Built on the host at
// plan time, read by every kernel of the forward and adjoint transforms.
struct BandDev {
    int64_t n;         // oversampled FFT length n_m = 2 N_m (0: band has no grid)
    int64_t Nm;        // NFFT bandwidth N_m (power of two >= K)
    int64_t K;         // frequencies 0..K-1 carry nonzero weight
    int64_t grid_off;  // element offset of the band's grids (nrhs x n) in the grid buffer
    int64_t D_off;     // element offset of the band's weight table (nrhs x K)
    int nrhs;          // right-hand sides: q for interpolated bands, 1 for Y_M
    int log2n;
    int route;         // 0 empty, 1 NFFT, 2 direct sum
    int dld;           // 0: weights D[s K + k]; > 0 (real exponents): one row of
                       // dld >= nrhs entries per exponent, D[k dld + s], zero-padded
    double yc, yh;     // band Y_m = [yc - yh, yc + yh] (paper's y), for barycentric weights
    double yh_inv;     // 1 / yh (a power of two times 1/y_1)
    int64_t node_off;  // first node of the band in sorted order
    int64_t dslot;     // direct route: offset of the band's partial sums (nodes x nchunk)
    int nchunk;        // direct route: coefficient chunks
    int pad2;
    int64_t c_off;     // offset of the band's transform in the coefficient buffer (batches)
    int64_t nodes;     // nodes of the band (sorted positions node_off .. node_off + nodes)
    // real exponents (NNFFT bands): 2 xc is the integer grid position of the
    // band's centre frequency, gh the half-width of the occupied grid
    // frequencies, phi_off the offset of the grid's 1/Phi table
    double xc;
    int64_t gh;
    int64_t phi_off;
    // window gather fused into the FFT's second pass (FP32 forward, four-step
    // grids whose nodes are few for the grid): the grid is never written;
    // pass 2 leaves per-node partial tap sums instead (see k_pass2)
    int fused;         // 1: this band's gather is fused into pass 2
    int pparts;        // partial sums per node and right-hand side (row blocks a window spans)
    int64_t ent_off;   // first entry of the band's (node, row block) entry list
    int64_t rbs_off;   // offset of the band's row-block starts (n2 / rows-per-CTA + 1 of them)
    int64_t pp_off;    // offset of the band's partial sums (nrhs x nodes x pparts complex)
    int64_t ph_off;    // offset (in float4) of the band's entry window values
    // Oversampling below 2: a band whose frequencies 0..K-1 are split into
    // nsub contiguous sub-bands, each its own NFFT on a power-of-two grid of
    // n = sigma K_p points (sigma < 2).  The band keeps its nodes (band ids
    // point to it) but has no grid; its sub-bands are bands[sub0 ..
    // sub0 + nsub) with parent = the band, frequencies k0 .. k0 + K - 1, the
    // band's nodes, and the centre frequency k0 + Nm/2.  A split band's n,
    // log2n and kb are its sub-bands' (the grid of the node cells).
    int64_t k0;        // first frequency of a sub-band (0 otherwise)
    int nsub;          // > 0: split band (no grid of its own)
    int sub0;          // first sub-band of a split band
    int parent;        // sub-band: its band; -1 otherwise
    int pad3;
    double kb;         // Kaiser-Bessel shape b = pi (2 - 1/sigma) of this band's grid
};

// ---------------------------------------------------------------------------
// Shared-memory Stockham FFT, radix 8/4/2, 8 elements per thread.
//
// Computes X[l] = sum_i x[i] exp(SIGN * 2 pi i * i l / L) in place on a
// smem array holding element i at pad8(i), L = 2^log2L (8 <= L), using nthr = L/8
// threads numbered t = 0..nthr-1.  Each stage with radix R, span Ns takes
// job jj = (R-point butterfly) reading x[jj + r L/R], twiddling by
// w^(r k), w = exp(SIGN 2 pi i / (Ns R)), k = jj mod Ns, and writing to
// (jj - k) R + k + r Ns: the self-sorting Stockham order, so the result is in
// natural order.  Every thread of the block must call it (it synchronises).

// Padded shared-memory index: one spare element after every 8.  The Stockham
// stores of the first stages have strides that are multiples of 8 elements and
// would fall on two banks; with the pad they spread over all of them.  A
// buffer for L points needs padded_len(L) elements.
__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }
__host__ __device__ __forceinline__ int padded_len(int L) { return L + (L >> 3); }

template <int SIGN, typename C> __device__ __forceinline__ C mul_i(C a) {
    // a * (SIGN * i)
    return SIGN > 0 ? C{-a.y, a.x} : C{a.y, -a.x};
}

template <int SIGN, typename C> __device__ __forceinline__ void dft2(C& a0, C& a1) {
    C t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <int SIGN, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C u0 = cadd(a0, a2), u1 = csub(a0, a2);
    C u2 = cadd(a1, a3), u3 = mul_i<SIGN>(csub(a1, a3));
    a0 = cadd(u0, u2);
    a2 = csub(u0, u2);
    a1 = cadd(u1, u3);
    a3 = csub(u1, u3);
}

template <int SIGN, typename T> __device__ __forceinline__ void dft8(C_t<T>* a) {
    using C = C_t<T>;
    const T h = (T)0.70710678118654752440084436210485;
    C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<SIGN>(e0, e1, e2, e3);
    dft4<SIGN>(o0, o1, o2, o3);
    // o1 *= w8, o2 *= w8^2 = SIGN i, o3 *= w8^3, w8 = (1 + SIGN i)/sqrt 2
    C t1 = {(o1.x - SIGN * o1.y) * h, (o1.y + SIGN * o1.x) * h};
    C t2 = mul_i<SIGN>(o2);
    C t3 = {(-o3.x - SIGN * o3.y) * h, (-o3.y + SIGN * o3.x) * h};
    a[0] = cadd(e0, o0);
    a[4] = csub(e0, o0);
    a[1] = cadd(e1, t1);
    a[5] = csub(e1, t1);
    a[2] = cadd(e2, t2);
    a[6] = csub(e2, t2);
    a[3] = cadd(e3, t3);
    a[7] = csub(e3, t3);
}

template <int R, int SIGN, typename T>
__device__ __forceinline__ void fft_stage(C_t<T>* buf, int L, int Ns, int t, int nthr, bool active) {
    using C = C_t<T>;
    constexpr int J = 8 / R;
    C v[8];
    const T inv_span = (T)1 / (T)(Ns * R);   // a power of two
    if (active) {
#pragma unroll
        for (int jb = 0; jb < J; ++jb) {
            const int jj = t + jb * nthr;
            const int k = jj & (Ns - 1);
#pragma unroll
            for (int r = 0; r < R; ++r) v[jb * R + r] = buf[pad8(jj + r * (L / R))];
            if (Ns > 1) {
                // k < Ns and 1/(Ns R) is a power of two: exact argument
                C w1 = expipi<T>((T)(2 * SIGN) * (T)k * inv_span);
                C w = w1;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    v[jb * R + r] = cmul(v[jb * R + r], w);
                    w = cmul(w, w1);
                }
            }
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int jb = 0; jb < J; ++jb) {
            C* a = v + jb * R;
            if (R == 8) dft8<SIGN, T>(a);
            if (R == 4) dft4<SIGN>(a[0], a[1], a[2], a[3]);
            if (R == 2) dft2<SIGN>(a[0], a[1]);
            const int jj = t + jb * nthr;
            const int k = jj & (Ns - 1);
            const int base = (jj - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[pad8(base + r * Ns)] = a[r];
        }
    }
    __syncthreads();
}

template <int SIGN, typename T>
__device__ __forceinline__ void fft_smem(C_t<T>* buf, int log2L, int t, bool active) {
    const int L = 1 << log2L;
    const int nthr = L >> 3;
    int Ns = 1, rem = log2L;
    while (rem >= 3) {
        fft_stage<8, SIGN, T>(buf, L, Ns, t, nthr, active);
        Ns <<= 3;
        rem -= 3;
    }
    if (rem == 2) fft_stage<4, SIGN, T>(buf, L, Ns, t, nthr, active);
    if (rem == 1) fft_stage<2, SIGN, T>(buf, L, Ns, t, nthr, active);
}

}  // namespace fl
