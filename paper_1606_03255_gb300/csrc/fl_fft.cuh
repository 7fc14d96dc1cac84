// fl_fft.cuh -- the FFTs of the band grids (the "FFT" step of every NFFT in
// Algorithm 2 of Kunis & Melzer), shared by fl_fft_f32.cu and fl_fft_f64.cu.
//
// * prep_value: the forward input of a band grid, c_k D[s][k] at the grid index
//   of the centred frequency k' = k - N_m/2 (deconvolution and Lagrange /
//   coupling weights are folded into D), zero elsewhere.
// * fft_ct: shared-memory Stockham FFT with the length a compile-time constant,
//   radix 8 (then 4 or 2), 8 elements per thread, every stage unrolled.
// * k_pass1 / k_pass2: the two passes of the four-step FFT of length
//   n = n1 n2 for grids above one CTA (n > 4096).
#pragma once

#include "fl_plan.cuh"

namespace fl {

constexpr double kTwoPiFFT = 6.283185307179586476925286766559;

// Forward input: grid index i in [0, n) holds frequency k' = i (i < n/2) or
// i - n, i.e. k = k' + N_m/2; value c_k D[s][k] for 0 <= k < K, else 0.
template <typename T, bool DERIV>
__device__ __forceinline__ C_t<T> prep_value(int64_t i, const BandDev& B, int s,
                                             const C_t<T>* __restrict__ c,
                                             const T* __restrict__ D) {
    const int64_t kp = (i < (B.n >> 1)) ? i : i - B.n;
    const int64_t k = kp + (B.Nm >> 1);
    if (k < 0 || k >= B.K) return C_t<T>{(T)0, (T)0};
    const T d = D[B.D_off + (int64_t)s * B.K + k];
    C_t<T> v = c[k];
    if (DERIV) {   // (2 pi i k) c_k
        const T w = (T)(kTwoPiFFT * (double)k);
        v = C_t<T>{-v.y * w, v.x * w};
    }
    return C_t<T>{v.x * d, v.y * d};
}

// Same with 32-bit grid indices and the band's c/D base pointers resolved.
template <typename T, bool DERIV>
__device__ __forceinline__ C_t<T> prep_value32(int i, int n, int half_Nm, int K,
                                               const C_t<T>* __restrict__ c,
                                               const T* __restrict__ Ds) {
    const int kp = (i < (n >> 1)) ? i : i - n;
    const int k = kp + half_Nm;
    if (k < 0 || k >= K) return C_t<T>{(T)0, (T)0};
    const T d = Ds[k];
    C_t<T> v = c[k];
    if (DERIV) {
        const T w = (T)(kTwoPiFFT * (double)k);
        v = C_t<T>{-v.y * w, v.x * w};
    }
    return C_t<T>{v.x * d, v.y * d};
}

// ---------------------------------------------------------------------------
// Compile-time-length Stockham FFT (same transform as fft_smem).

template <int R, int NS, int L, int SIGN, typename T>
__device__ __forceinline__ void fft_stage_ct(C_t<T>* buf, int t) {
    using C = C_t<T>;
    constexpr int J = 8 / R;
    constexpr int NTHR = L / 8;
    C v[8];
#pragma unroll
    for (int jb = 0; jb < J; ++jb) {
        const int jj = t + jb * NTHR;
        const int k = jj & (NS - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) v[jb * R + r] = buf[pad8(jj + r * (L / R))];
        if constexpr (NS > 1) {
            // k < NS and 1/(NS R) is a power of two: exact argument
            const C w1 = expipi<T>((T)(2 * SIGN) * (T)k * (T)(1.0 / (NS * R)));
            C w = w1;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                v[jb * R + r] = cmul(v[jb * R + r], w);
                w = cmul(w, w1);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int jb = 0; jb < J; ++jb) {
        C* a = v + jb * R;
        if constexpr (R == 8) dft8<SIGN, T>(a);
        if constexpr (R == 4) dft4<SIGN>(a[0], a[1], a[2], a[3]);
        if constexpr (R == 2) dft2<SIGN>(a[0], a[1]);
        const int jj = t + jb * NTHR;
        const int k = jj & (NS - 1);
        const int base = (jj - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad8(base + r * NS)] = a[r];
    }
    __syncthreads();
}

template <int LOG2L, int SIGN, typename T, int DONE = 0>
__device__ __forceinline__ void fft_ct(C_t<T>* buf, int t) {
    constexpr int L = 1 << LOG2L;
    if constexpr (LOG2L - DONE >= 3) {
        fft_stage_ct<8, (1 << DONE), L, SIGN, T>(buf, t);
        fft_ct<LOG2L, SIGN, T, DONE + 3>(buf, t);
    } else if constexpr (LOG2L - DONE == 2) {
        fft_stage_ct<4, (1 << DONE), L, SIGN, T>(buf, t);
    } else if constexpr (LOG2L - DONE == 1) {
        fft_stage_ct<2, (1 << DONE), L, SIGN, T>(buf, t);
    }
}

// Columns (pass 1) or rows (pass 2) per CTA: >= 64 contiguous bytes per global
// row segment, <= 1024 threads (len/8 per FFT).
template <typename T, int LOG2L>
struct PassTile {
    static constexpr int L = 1 << LOG2L;
    static constexpr int W0 = (int)(64 / sizeof(C_t<T>));
    static constexpr int TILES = (W0 * (L / 8) <= 1024) ? W0 : (1024 / (L / 8));
    static constexpr int LOG2T = TILES == 8 ? 3 : TILES == 4 ? 2 : TILES == 2 ? 1 : 0;
    static constexpr int NT = TILES * (L / 8);
    // padded length + an offset that puts consecutive tiles P/TILES bank
    // groups apart (P = 128 bytes / element size), so the transposing
    // load/store loops (consecutive threads on consecutive tiles) spread over
    // the banks
    static constexpr int P = (int)(128 / sizeof(C_t<T>));
    static constexpr int LD = L + (L >> 3) + (TILES >= P ? 1 : P / TILES);
    static constexpr size_t SMEM = (size_t)TILES * LD * sizeof(C_t<T>);
    // 2048 resident threads for float (32 registers), 1024 for double
    static constexpr int MINB = (sizeof(T) == 4 ? 2048 : 1024) / NT;
};

// Pass 1 for a tile of TILES columns i1 of one right-hand side s: the
// length-n2 FFTs over i2 of x[i1 + n1 i2], twiddled by exp(SIGN 2 pi i i1 l2/n),
// stored to Y[l2 n1 + i1].  MODE 0: x generated by prep_value (forward);
// MODE 1: x read from the band grid (adjoint).
template <typename T, int SIGN, int MODE, bool DERIV, int LOG2L>
__global__ void __launch_bounds__(PassTile<T, LOG2L>::NT, PassTile<T, LOG2L>::MINB)
    k_pass1(BandDev B, int rhs0, int log2n1, const C_t<T>* __restrict__ c,
            const T* __restrict__ D, const C_t<T>* __restrict__ src, C_t<T>* __restrict__ Y) {
    using C = C_t<T>;
    using PT = PassTile<T, LOG2L>;
    constexpr int L = PT::L, TC = PT::TILES, NT = PT::NT, LD = PT::LD;
    extern __shared__ unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int n1 = 1 << log2n1;
    const int n = n1 << LOG2L;
    const int s = rhs0 + blockIdx.y;
    const int i1b = blockIdx.x * TC;
    const int tid = threadIdx.x;
    if constexpr (MODE == 0) {
        const T* Ds = D + B.D_off + (int64_t)s * B.K;
        const int K = (int)B.K, half = (int)(B.Nm >> 1);
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int idx = tid + it * NT;
            const int col = idx & (TC - 1), i2 = idx >> PT::LOG2T;
            sm[col * LD + pad8(i2)] =
                prep_value32<T, DERIV>(i1b + col + (i2 << log2n1), n, half, K, c, Ds);
        }
    } else {
        const C* in = src + B.grid_off + (int64_t)s * n;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int idx = tid + it * NT;
            const int col = idx & (TC - 1), i2 = idx >> PT::LOG2T;
            sm[col * LD + pad8(i2)] = in[i1b + col + (i2 << log2n1)];
        }
    }
    __syncthreads();
    fft_ct<LOG2L, SIGN, T>(sm + (tid / (L / 8)) * LD, tid & (L / 8 - 1));
    // twiddles exp(SIGN 2 pi i i1 l2 / n) by recurrence along this thread's l2
    const int col = tid & (TC - 1);
    const int l20 = tid >> PT::LOG2T;
    constexpr int S = NT / TC;                    // = L/8, the l2 step between iterations
    const int i1 = i1b + col;
    const T inv_n = (T)1 / (T)n;                  // a power of two
    int e0 = i1 * l20;                            // < n
    if (e0 >= n / 2) e0 -= n;
    int es = (i1 * S) & (n - 1);
    if (es >= n / 2) es -= n;
    C w = expipi<T>((T)(2 * SIGN) * (T)e0 * inv_n);
    const C step = expipi<T>((T)(2 * SIGN) * (T)es * inv_n);
    C* out = Y + (int64_t)blockIdx.y * n;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int l2 = l20 + it * S;
        out[(int64_t)l2 * n1 + i1] = cmul(sm[col * LD + pad8(l2)], w);
        w = cmul(w, step);
    }
}

// Pass 2 for a tile of TILES rows l2: the length-n1 FFTs over i1 of
// Y[l2 n1 + i1], stored to X[l2 + n2 l1] (natural order of the length-n
// transform) in the band grid.
template <typename T, int SIGN, int LOG2L>
__global__ void __launch_bounds__(PassTile<T, LOG2L>::NT, PassTile<T, LOG2L>::MINB)
    k_pass2(BandDev B, int rhs0, int log2n2, const C_t<T>* __restrict__ Y, C_t<T>* __restrict__ dst) {
    using C = C_t<T>;
    using PT = PassTile<T, LOG2L>;
    constexpr int L = PT::L, TR = PT::TILES, NT = PT::NT, LD = PT::LD;
    extern __shared__ unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int n = L << log2n2;
    const int s = rhs0 + blockIdx.y;
    const int l2b = blockIdx.x * TR;
    const int tid = threadIdx.x;
    const C* in = Y + (int64_t)blockIdx.y * n + (int64_t)l2b * L;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int idx = tid + it * NT;
        const int row = idx >> LOG2L, i1 = idx & (L - 1);
        sm[row * LD + pad8(i1)] = in[idx];
    }
    __syncthreads();
    fft_ct<LOG2L, SIGN, T>(sm + (tid / (L / 8)) * LD, tid & (L / 8 - 1));
    C* out = dst + B.grid_off + (int64_t)s * n + l2b;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int idx = tid + it * NT;
        const int row = idx & (TR - 1), l1 = idx >> PT::LOG2T;
        out[row + ((int64_t)l1 << log2n2)] = sm[row * LD + pad8(l1)];
    }
}

// Host launchers of one band's passes for right-hand sides rhs0..rhs0+ns-1;
// the pass length picks the compiled instantiation.

template <typename T, int SIGN, int MODE, bool DERIV, int LOG2L>
static cudaError_t pass1_ct(const BandDev& B, int rhs0, int ns, int log2n1, const C_t<T>* c,
                            const T* D, const C_t<T>* src, C_t<T>* Y, cudaStream_t st) {
    using PT = PassTile<T, LOG2L>;
    auto k = k_pass1<T, SIGN, MODE, DERIV, LOG2L>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PT::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    k<<<dim3((unsigned)((1 << log2n1) / PT::TILES), (unsigned)ns), PT::NT, PT::SMEM, st>>>(
        B, rhs0, log2n1, c, D, src, Y);
    return cudaGetLastError();
}

template <typename T, int SIGN, int LOG2L>
static cudaError_t pass2_ct(const BandDev& B, int rhs0, int ns, int log2n2, const C_t<T>* Y,
                            C_t<T>* dst, cudaStream_t st) {
    using PT = PassTile<T, LOG2L>;
    auto k = k_pass2<T, SIGN, LOG2L>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PT::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    k<<<dim3((unsigned)((1 << log2n2) / PT::TILES), (unsigned)ns), PT::NT, PT::SMEM, st>>>(
        B, rhs0, log2n2, Y, dst);
    return cudaGetLastError();
}

// Pass 1 (length n2 = 2^log2n2, 6..12) over all n1 = 2^log2n1 columns.
template <typename T, int SIGN, int MODE, bool DERIV>
cudaError_t launch_pass1(const BandDev& B, int rhs0, int ns, int log2n1, int log2n2,
                         const C_t<T>* c, const T* D, const C_t<T>* src, C_t<T>* Y,
                         cudaStream_t st) {
    switch (log2n2) {
#define FL_P1(LG) \
    case LG: return pass1_ct<T, SIGN, MODE, DERIV, LG>(B, rhs0, ns, log2n1, c, D, src, Y, st);
        FL_P1(6) FL_P1(7) FL_P1(8) FL_P1(9) FL_P1(10) FL_P1(11) FL_P1(12)
#undef FL_P1
        default: return cudaErrorInvalidValue;
    }
}

// Pass 2 (length n1 = 2^log2n1, 7..12) over all n2 = 2^log2n2 rows.
template <typename T, int SIGN>
cudaError_t launch_pass2(const BandDev& B, int rhs0, int ns, int log2n1, int log2n2,
                         const C_t<T>* Y, C_t<T>* dst, cudaStream_t st) {
    switch (log2n1) {
#define FL_P2(LG) \
    case LG: return pass2_ct<T, SIGN, LG>(B, rhs0, ns, log2n2, Y, dst, st);
        FL_P2(6) FL_P2(7) FL_P2(8) FL_P2(9) FL_P2(10) FL_P2(11) FL_P2(12)
#undef FL_P2
        default: return cudaErrorInvalidValue;
    }
}

#define FL_FFT_EXTERN(T)                                                                    \
    extern template cudaError_t launch_pass1<T, 1, 0, false>(const BandDev&, int, int, int, int, \
                                                             const C_t<T>*, const T*,         \
                                                             const C_t<T>*, C_t<T>*,          \
                                                             cudaStream_t);                   \
    extern template cudaError_t launch_pass1<T, 1, 0, true>(const BandDev&, int, int, int, int,  \
                                                            const C_t<T>*, const T*,          \
                                                            const C_t<T>*, C_t<T>*,           \
                                                            cudaStream_t);                    \
    extern template cudaError_t launch_pass1<T, -1, 1, false>(const BandDev&, int, int, int,     \
                                                              int, const C_t<T>*, const T*,   \
                                                              const C_t<T>*, C_t<T>*,         \
                                                              cudaStream_t);                  \
    extern template cudaError_t launch_pass2<T, 1>(const BandDev&, int, int, int, int,          \
                                                   const C_t<T>*, C_t<T>*, cudaStream_t);     \
    extern template cudaError_t launch_pass2<T, -1>(const BandDev&, int, int, int, int,         \
                                                    const C_t<T>*, C_t<T>*, cudaStream_t);

}  // namespace fl
