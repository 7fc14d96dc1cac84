// fl_fft.cuh -- the FFTs of the band grids (the "FFT" step of every NFFT in
// Algorithm 2 of Kunis & Melzer), shared by fl_fft_f32.cu and fl_fft_f64.cu.
//
// * prep_value: the forward input of a band grid, c_k D[s][k] at the grid index
//   of the centred frequency k' = k - N_m/2 (deconvolution and Lagrange /
//   coupling weights are folded into D), zero elsewhere.
// * fft_ct: shared-memory Stockham FFT with the length a compile-time constant,
//   radix 16 (then 8, 4 or 2), 16 elements per thread, every stage unrolled,
//   XOR-swizzled shared memory.
// * k_pass1 / k_pass2: the two passes of the four-step FFT of length
//   n = n1 n2 for grids above one CTA (n > 4096).
#pragma once

#include <type_traits>

#include "fl_plan.cuh"

namespace fl {

constexpr double kTwoPiFFT = 6.283185307179586476925286766559;

// 2 pi k in T: float from the exact float k (k < 2^24), with one rounding and
// no FP64 arithmetic; double (and float pairs) through double.
template <typename T> __device__ __forceinline__ T deriv_weight(int64_t k) {
    if constexpr (sizeof(T) == 4) return (float)k * 6.28318530717958647692f;
    else return (T)(kTwoPiFFT * (double)k);
}

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
    if (DERIV) {   // (2 pi i k) c_k at the global frequency; float: k < 2^24 exact, one rounding
        const T w = deriv_weight<T>(k + B.k0);
        v = C_t<T>{-v.y * w, v.x * w};
    }
    return C_t<T>{v.x * d, v.y * d};
}

// Same with 32-bit grid indices and the band's c/D base pointers resolved, for
// an element of pass-1 row r: the row holds grid indices i in [r n/16,
// (r+1) n/16), so whether i is a negative centred frequency (i >= n/2) is
// known at compile time (HI = r >= 8) and k = i (- n) + N_m/2 lies in the band
// iff 0 <= k < K, one unsigned comparison.  Branch-free: outside the band the
// loads read index 0 (in bounds, so a thread's loads can all be in flight
// together) and the weight is replaced by zero.  k0: the band's first
// frequency (sub-bands; c is already offset by it).
template <typename T, bool DERIV, bool HI>
__device__ __forceinline__ C_t<T> prep_value32(int i, int n, int half_Nm, int K, int k0,
                                               const C_t<T>* __restrict__ c,
                                               const T* __restrict__ Ds) {
    const int k = HI ? i - n + half_Nm : i + half_Nm;
    const bool in = (unsigned)k < (unsigned)K;
    const int kk = in ? k : 0;
    const T dl = Ds[kk];
    const T d = in ? dl : (T)0;
    C_t<T> v = c[kk];
    if (DERIV) {
        const T w = deriv_weight<T>(kk + k0);
        v = C_t<T>{-v.y * w, v.x * w};
    }
    return C_t<T>{v.x * d, v.y * d};
}

// ---------------------------------------------------------------------------
// Compile-time-length Stockham FFT, radix 16 (then 8, 4 or 2), 16 elements per
// thread.  Same transform and stage structure as fft_smem: stage (R, NS) takes
// job jj reading x[jj + r L/R], twiddling by w^(r k), w = exp(SIGN 2 pi i /
// (NS R)), k = jj mod NS, and writing to (jj - k) R + k + r NS.
//
// Shared-memory layout: element e lives at swz(e) = e ^ ((e >> 4) & (P - 1)),
// P = 128 bytes / element size (16 for float2, 8 for double2).  The XOR keeps
// aligned runs of 16 contiguous elements a permutation of one bank row and
// spreads the stride-16 stores of the first stage (e = 16 j + r) over P banks,
// so every stage's loads and stores are free of bank conflicts.

template <typename T> __device__ __forceinline__ int swz(int e) {
    constexpr int P = (int)(128 / sizeof(C_t<T>));
    return e ^ ((e >> 4) & (P - 1));
}

// swz(b0 + r D) from bs = swz(b0) for a stride D that is a multiple of 16 and a
// base b0 whose bits below log2(D) hold everything b0 has below the top part
// (the load pattern jj + r L/R with jj < L/R, and the store pattern
// (jj - k) R + k + r NS with k < NS): the mask (e >> 4) & (P - 1) of
// e = b0 + r D is then mask(b0) ^ ((r D >> 4) & (P - 1)) with disjoint bits,
// and the XOR touches only bits below 4, so
//   swz(b0 + r D) = (swz(b0) ^ ((r D >> 4) & (P - 1))) + r D,
// a compile-time XOR constant and offset per unrolled r.
template <typename T, int D> __device__ __forceinline__ int swz_step(int bs, int r) {
    constexpr int P = (int)(128 / sizeof(C_t<T>));
    static_assert(D % 16 == 0, "stride of the swizzle shortcut");
    return (bs ^ (((r * D) >> 4) & (P - 1))) + r * D;
}

// 16-point DFT in registers (4 x 4 with internal twiddles), sign SIGN.
template <int SIGN, typename T> __device__ __forceinline__ void dft16(C_t<T>* a) {
    using C = C_t<T>;
    const T c1 = (T)0.92387953251128675612818318939679;   // cos(pi/8)
    const T s1 = (T)0.38268343236508977172845998403040;   // sin(pi/8)
    const T h = (T)0.70710678118654752440084436210485;
#pragma unroll
    for (int b = 0; b < 4; ++b) dft4<SIGN>(a[b], a[4 + b], a[8 + b], a[12 + b]);
    // a[b + 4 k1] *= W16^(b k1), W16 = exp(SIGN 2 pi i / 16)
    a[5] = cmul(a[5], C{c1, SIGN * s1});      // W^1
    a[6] = cmul(a[6], C{h, SIGN * h});        // W^2
    a[7] = cmul(a[7], C{s1, SIGN * c1});      // W^3
    a[9] = cmul(a[9], C{h, SIGN * h});        // W^2
    a[10] = mul_i<SIGN>(a[10]);               // W^4
    a[11] = cmul(a[11], C{-h, SIGN * h});     // W^6
    a[13] = cmul(a[13], C{s1, SIGN * c1});    // W^3
    a[14] = cmul(a[14], C{-h, SIGN * h});     // W^6
    a[15] = cmul(a[15], C{-c1, -SIGN * s1});  // W^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<SIGN>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
    // now a[4 k1 + k2] = X[k1 + 4 k2]: transpose to natural order
    C t;
    t = a[1]; a[1] = a[4]; a[4] = t;
    t = a[2]; a[2] = a[8]; a[8] = t;
    t = a[3]; a[3] = a[12]; a[12] = t;
    t = a[6]; a[6] = a[9]; a[9] = t;
    t = a[7]; a[7] = a[13]; a[13] = t;
    t = a[11]; a[11] = a[14]; a[14] = t;
}

// Twiddles w^r, r = 0..R-1, of w = exp(i pi x): w and w^4 from sincospi, the
// rest as products of at most three factors (errors stay a few ulps).
template <int R, typename T>
__device__ __forceinline__ void twiddle_powers(T x, C_t<T>* w) {
    using C = C_t<T>;
    w[0] = C{(T)1, (T)0};
    const C w1 = expipi<T>(x);
    w[1] = w1;
    if constexpr (R >= 4) {
        w[2] = cmul(w1, w1);
        w[3] = cmul(w[2], w1);
    }
    if constexpr (R >= 8) {
        const C w4 = expipi<T>((T)4 * x);
        w[4] = w4;
#pragma unroll
        for (int b = 1; b < 4; ++b) w[4 + b] = cmul(w4, w[b]);
        if constexpr (R == 16) {
            const C w8 = cmul(w4, w4);
            const C w12 = cmul(w8, w4);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                w[8 + b] = b ? cmul(w8, w[b]) : w8;
                w[12 + b] = b ? cmul(w12, w[b]) : w12;
            }
        }
    }
}

// Stage twiddles come from the plan-time table laid out by tw_region / tw_off
// (fl_common.cuh); SIGN = -1 takes the conjugate.
// The twiddle pair at p (entries p[0], p[1]): one 16-byte load in float.
template <int SIGN> __device__ __forceinline__ void tw_load2(const float2* p, float2& a, float2& b) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    a = float2{q.x, SIGN < 0 ? -q.y : q.y};
    b = float2{q.z, SIGN < 0 ? -q.w : q.w};
}
template <int SIGN> __device__ __forceinline__ void tw_load2(const double2* p, double2& a, double2& b) {
    a = __ldg(p);
    b = __ldg(p + 1);
    if (SIGN < 0) {
        a.y = -a.y;
        b.y = -b.y;
    }
}

template <int SIGN> __device__ __forceinline__ void tw_load2(const ffc* p, ffc& a, ffc& b) {
    const float4 qa = __ldg(reinterpret_cast<const float4*>(p));
    const float4 qb = __ldg(reinterpret_cast<const float4*>(p + 1));
    a = ffc{ff(qa.x, qa.y), SIGN < 0 ? ff(-qa.z, -qa.w) : ff(qa.z, qa.w)};
    b = ffc{ff(qb.x, qb.y), SIGN < 0 ? ff(-qb.z, -qb.w) : ff(qb.z, qb.w)};
}

// Float pairs: exp(SIGN 2 pi i e / 2^24), 0 <= e < 2^24, as the product of two
// plan-time table entries (each rounded once from FP64): tab[a] = exp(2 pi i
// a / 2^12) and tab[4096 + b] = exp(2 pi i b / 2^24), e = 2^12 a + b.
template <int SIGN> __device__ __forceinline__ ffc ff_twiddle24(const ffc* __restrict__ tab, int e) {
    const float4 qa = __ldg(reinterpret_cast<const float4*>(tab + (e >> 12)));
    const float4 qb = __ldg(reinterpret_cast<const float4*>(tab + 4096 + (e & 4095)));
    const ffc w = cmul(ffc{ff(qa.x, qa.y), ff(qa.z, qa.w)}, ffc{ff(qb.x, qb.y), ff(qb.z, qb.w)});
    return SIGN < 0 ? ffc{w.x, -w.y} : w;
}

// v[1 .. R-1] *= w^(r k) from the stage table tws (pairs, see fl_common.cuh).
template <int R, int NS, int SIGN, typename C>
__device__ __forceinline__ void apply_stage_twiddles(C* v, const C* __restrict__ tws, int k) {
    const C* tk = tws + 2 * k;
#pragma unroll
    for (int p = 0; p < R / 2; ++p) {
        C w1, w2;
        tw_load2<SIGN>(tk + p * 2 * NS, w1, w2);
        v[2 * p + 1] = cmul(v[2 * p + 1], w1);
        if (2 * p + 2 < R) v[2 * p + 2] = cmul(v[2 * p + 2], w2);
    }
}

template <int R, int NS, int L, int SIGN, typename T>
__device__ __forceinline__ void fft16_stage(C_t<T>* buf, int t, const C_t<T>* __restrict__ tws) {
    using C = C_t<T>;
    constexpr int J = 16 / R;
    constexpr int NTHR = L / 16;
    C v[16];
#pragma unroll
    for (int jb = 0; jb < J; ++jb) {
        const int jj = t + jb * NTHR;
        const int k = jj & (NS - 1);
        if constexpr ((L / R) % 16 == 0) {
            const int bs = swz<T>(jj);
#pragma unroll
            for (int r = 0; r < R; ++r) v[jb * R + r] = buf[swz_step<T, L / R>(bs, r)];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[jb * R + r] = buf[swz<T>(jj + r * (L / R))];
        }
        if constexpr (NS > 1) apply_stage_twiddles<R, NS, SIGN>(v + jb * R, tws, k);
    }
    __syncthreads();
#pragma unroll
    for (int jb = 0; jb < J; ++jb) {
        C* a = v + jb * R;
        if constexpr (R == 16) dft16<SIGN, T>(a);
        if constexpr (R == 8) dft8<SIGN, T>(a);
        if constexpr (R == 4) dft4<SIGN>(a[0], a[1], a[2], a[3]);
        if constexpr (R == 2) dft2<SIGN>(a[0], a[1]);
        const int jj = t + jb * NTHR;
        const int k = jj & (NS - 1);
        const int base = (jj - k) * R + k;
        if constexpr (NS % 16 == 0) {
            const int bs = swz<T>(base);
#pragma unroll
            for (int r = 0; r < R; ++r) buf[swz_step<T, NS>(bs, r)] = a[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) buf[swz<T>(base + r * NS)] = a[r];
        }
    }
    __syncthreads();
}

// The same transform split so that its first stage can take its inputs from
// registers and its last stage can leave its outputs in registers: a first
// stage of radix 2^FIRST (16, or 8 with two butterflies per thread), radix-16
// middle stages, and a last stage of radix LAST_R.
template <int LOG2L, int FIRST = 4> struct StagePlan {
    static constexpr int REST = LOG2L - FIRST;                  // >= 1
    static constexpr int NSTAGE = 1 + (REST + 3) / 4;
    static constexpr int LAST_LOG = REST - 4 * ((REST + 3) / 4 - 1);   // 1..4
    static constexpr int LAST_R = 1 << LAST_LOG;
    static constexpr int LAST_NS = 1 << (LOG2L - LAST_LOG);
};

// First stage (radix 16, span 1) on v[r] = x[t + r L/16], stored to smem.
template <int LOG2L, int SIGN, typename T>
__device__ __forceinline__ void fft_first_from_regs(C_t<T>* v, C_t<T>* buf, int t) {
    dft16<SIGN, T>(v);
    // swz(16 t + r) = (16 t + mask) ^ r, mask = t & (P - 1) < 16
    const int bs = swz<T>(t * 16);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[bs ^ r] = v[r];
    __syncthreads();
}

// First stage as radix 8 (span 1) with the two butterflies jj = 2t and 2t + 1
// of one thread: v[8 b + r] = x[2t + b + r L/8].  Butterfly jj writes jj 8 + r,
// so the thread's 16 outputs are again the contiguous run 16 t .. 16 t + 15, and
// its inputs are 8 pairs of adjacent elements (16-byte loads for float).
template <int LOG2L, int SIGN, typename T>
__device__ __forceinline__ void fft_first8x2_from_regs(C_t<T>* v, C_t<T>* buf, int t) {
    dft8<SIGN, T>(v);
    dft8<SIGN, T>(v + 8);
    const int bs = swz<T>(t * 16);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[bs ^ r] = v[r];
    __syncthreads();
}

// Middle stages (radix 16, smem to smem) from span 2^DONE up to the last stage;
// twr = the twiddle table region of (LOG2L, FIRST).
template <int LOG2L, int FIRST, int SIGN, typename T, int DONE = FIRST>
__device__ __forceinline__ void fft_middle(C_t<T>* buf, int t, const C_t<T>* __restrict__ twr) {
    constexpr int L = 1 << LOG2L;
    if constexpr (DONE < LOG2L - StagePlan<LOG2L, FIRST>::LAST_LOG) {
        fft16_stage<16, (1 << DONE), L, SIGN, T>(buf, t, twr + tw_off(LOG2L, FIRST, DONE));
        fft_middle<LOG2L, FIRST, SIGN, T, DONE + 4>(buf, t, twr);
    }
}

// Last stage (radix LAST_R, span LAST_NS = L / LAST_R) from smem into
// registers: v[jb R + r] is output jj + r LAST_NS, jj = t + jb L/16.
template <int LOG2L, int FIRST, int SIGN, typename T>
__device__ __forceinline__ void fft_last_to_regs(const C_t<T>* buf, int t, C_t<T>* v,
                                                 const C_t<T>* __restrict__ twr) {
    using C = C_t<T>;
    using SP = StagePlan<LOG2L, FIRST>;
    constexpr int L = 1 << LOG2L, R = SP::LAST_R, NS = SP::LAST_NS, J = 16 / R, NTHR = L / 16;
    const C* tws = twr + tw_off(LOG2L, FIRST, LOG2L - SP::LAST_LOG);
#pragma unroll
    for (int jb = 0; jb < J; ++jb) {
        const int jj = t + jb * NTHR;   // < LAST_NS, so k = jj
        if constexpr ((L / R) % 16 == 0) {
            const int bs = swz<T>(jj);
#pragma unroll
            for (int r = 0; r < R; ++r) v[jb * R + r] = buf[swz_step<T, L / R>(bs, r)];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[jb * R + r] = buf[swz<T>(jj + r * (L / R))];
        }
        apply_stage_twiddles<R, NS, SIGN>(v + jb * R, tws, jj);
        C* a = v + jb * R;
        if constexpr (R == 16) dft16<SIGN, T>(a);
        if constexpr (R == 8) dft8<SIGN, T>(a);
        if constexpr (R == 4) dft4<SIGN>(a[0], a[1], a[2], a[3]);
        if constexpr (R == 2) dft2<SIGN>(a[0], a[1]);
    }
}

template <typename T> struct PassBudget {
    static constexpr int P1 = sizeof(T) == 4 ? FL_P1_THREADS_F32 : FL_P1_THREADS_F64;
    static constexpr int P2 = sizeof(T) == 4 ? FL_P2_THREADS_F32 : FL_P2_THREADS_F64;
};

// Columns (pass 1) or rows (pass 2) per CTA: pass_tiles (fl_plan.cuh).
// FL_PASS_REGT_F32: threads per SM the FP32 passes' register budget is sized
// for (65536 registers / this = registers per thread).
// FL_PASS_CARVEOUT: the passes' preferred shared-memory carveout in percent
// of the SM's shared/L1 storage (-1: pass_carveout below).
#ifndef FL_PASS_CARVEOUT
#define FL_PASS_CARVEOUT -1
#endif
#ifndef FL_PASS_REGT_F32
#define FL_PASS_REGT_F32 1024
#endif
template <typename T, int LOG2L, int TMAX, int SEG = 64>
struct PassTile {
    static constexpr int L = 1 << LOG2L;
    static constexpr int EPT = 16;                       // elements per thread
    static constexpr int TILES = pass_tiles((int)sizeof(C_t<T>), LOG2L, TMAX, SEG);
    static constexpr int LOG2T = TILES == 32 ? 5 : TILES == 16 ? 4 : TILES == 8 ? 3 : TILES == 4 ? 2
                                 : TILES == 2 ? 1 : 0;
    static_assert(TILES == 1 || TILES == 2 || TILES == 4 || TILES == 8 || TILES == 16 || TILES == 32,
                  "tile count");
    static constexpr int NT = TILES * (L / EPT);
    // offset between tiles: P/TILES bank groups (P = 128 bytes / element
    // size), so the transposing load/store loops (consecutive threads on
    // consecutive tiles) spread over the banks
    static constexpr int P = (int)(128 / sizeof(C_t<T>));
    static constexpr int LD = L + (TILES >= P ? 1 : P / TILES);
    static constexpr size_t SMEM = (size_t)TILES * LD * sizeof(C_t<T>);
    // register budget: 64 per thread for float (1024 threads per SM), 128 for
    // double (512)
    static constexpr int REGT = sizeof(T) == 4 ? FL_PASS_REGT_F32 : 512;
    static constexpr int MINB = (REGT / NT) > 0 ? (REGT / NT) : 1;
};

// Pass 1 for a tile of TILES columns i1 of one right-hand side s: the
// length-n2 FFTs over i2 of x[i1 + n1 i2], twiddled by exp(SIGN 2 pi i i1 l2/n),
// stored to Y[l2 n1 + i1].  MODE 0: x generated by prep_value (forward);
// MODE 1: x read from the band grid (adjoint).
template <typename T, int SIGN, int MODE, bool DERIV, int LOG2L>
__global__ void __launch_bounds__(PassTile<T, LOG2L, PassBudget<T>::P1, FL_P1_SEG_BYTES>::NT,
                                  PassTile<T, LOG2L, PassBudget<T>::P1, FL_P1_SEG_BYTES>::MINB)
    k_pass1(const PassItem* __restrict__ items, const BandDev* __restrict__ bands, int log2n1,
            const C_t<T>* __restrict__ c, const T* __restrict__ D, const C_t<T>* __restrict__ src,
            C_t<T>* __restrict__ Y, const C_t<T>* __restrict__ tw) {
    using C = C_t<T>;
    using PT = PassTile<T, LOG2L, PassBudget<T>::P1, FL_P1_SEG_BYTES>;
    using SP = StagePlan<LOG2L>;
    constexpr int L = PT::L, TC = PT::TILES, LD = PT::LD;
    extern __shared__ unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const PassItem item = items[blockIdx.y];
    const BandDev B = bands[item.band];
    const int n1 = 1 << log2n1;
    const int n = n1 << LOG2L;
    const int s = item.rhs;
    // columns fastest: the warp's global accesses are TC-column segments
    const int col = threadIdx.x & (TC - 1);
    const int t = threadIdx.x >> PT::LOG2T;        // thread within the column FFT
    const int i1 = blockIdx.x * TC + col;
    C* buf = sm + col * LD;
    C v[16];
    if constexpr (MODE == 0) {
        const T* Ds = D + B.D_off + (int64_t)s * B.K;
        const int K = (int)B.K, half = (int)(B.Nm >> 1), k0 = (int)B.k0;
        // with sigma = 2 (half <= n/4 and K - half <= n/4), i2 = t + r L/16 in
        // [n2/4, 3 n2/4) (r = 4..11) holds grid indices in [n/4, 3n/4):
        // centred frequencies outside the band, always zero (a sub-band at
        // sigma < 2 reaches into them)
        const C* cb = c + B.c_off;
        const int i0 = i1 + (t << log2n1), di = (L / 16) << log2n1;   // row r: i0 + r di
        if (4 * half <= n && 4 * (K - half) <= n) {
#pragma unroll
            for (int r = 0; r < 16; ++r)
                v[r] = (r >= 4 && r < 12) ? C{(T)0, (T)0}
                       : r < 8 ? prep_value32<T, DERIV, false>(i0 + r * di, n, half, K, k0, cb, Ds)
                               : prep_value32<T, DERIV, true>(i0 + r * di, n, half, K, k0, cb, Ds);
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r)
                v[r] = r < 8 ? prep_value32<T, DERIV, false>(i0 + r * di, n, half, K, k0, cb, Ds)
                             : prep_value32<T, DERIV, true>(i0 + r * di, n, half, K, k0, cb, Ds);
        }
    } else {
        const C* in = src + B.grid_off + (int64_t)s * n;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = in[i1 + ((t + r * (L / 16)) << log2n1)];
    }
    const C* twr = tw + tw_region(LOG2L, 4);
    fft_first_from_regs<LOG2L, SIGN, T>(v, buf, t);
    fft_middle<LOG2L, 4, SIGN, T>(buf, t, twr);
    fft_last_to_regs<LOG2L, 4, SIGN, T>(buf, t, v, twr);
    // outputs l2 = jj + r NS, jj = t + jb L/16, twiddled by exp(SIGN 2 pi i i1 l2 / n)
    // = w0 rho^jb step^r with w0 = exp(.. i1 t), rho = exp(.. i1 L/16) and
    // step = exp(.. i1 NS): three sincospi values and short products
    constexpr int R = SP::LAST_R, NS = SP::LAST_NS, J = 16 / R;
    C* out = Y + item.y_off;
    if constexpr (std::is_same<T, ff>::value) {
        // float pairs: the same factorisation w0 rho^jb step^r as below, with
        // the base factors from the two plan-time tables after the stage table
        // (exponents i1 l2 < n <= 2^24, scaled to units of 2^-24 turns) and the
        // powers of step formed by products at most three deep
        const C* tab = tw + kTwEntries;
        const int sh = 24 - (log2n1 + LOG2L);
        C step[R];
        step[0] = C{ff(1), ff(0)};
        if constexpr (R >= 2) step[1] = ff_twiddle24<SIGN>(tab, ((i1 * NS) & (n - 1)) << sh);
        if constexpr (R >= 4) {
            step[2] = cmul(step[1], step[1]);
            step[3] = cmul(step[2], step[1]);
        }
        if constexpr (R >= 8) {
            step[4] = ff_twiddle24<SIGN>(tab, ((i1 * 4 * NS) & (n - 1)) << sh);
#pragma unroll
            for (int b = 1; b < 4; ++b) step[4 + b] = cmul(step[4], step[b]);
        }
        if constexpr (R == 16) {
            step[8] = ff_twiddle24<SIGN>(tab, ((i1 * 8 * NS) & (n - 1)) << sh);
            step[12] = ff_twiddle24<SIGN>(tab, ((i1 * 12 * NS) & (n - 1)) << sh);
#pragma unroll
            for (int b = 1; b < 4; ++b) {
                step[8 + b] = cmul(step[8], step[b]);
                step[12 + b] = cmul(step[12], step[b]);
            }
        }
#pragma unroll
        for (int jb = 0; jb < J; ++jb) {
            const int jj = t + jb * (L / 16);
            const C wj = ff_twiddle24<SIGN>(tab, (i1 * jj) << sh);   // i1 jj < n
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int l2 = jj + r * NS;
                out[(int64_t)l2 * n1 + i1] = cmul(v[jb * R + r], cmul(wj, step[r]));
            }
        }
    } else {
        const T inv_n = (T)1 / (T)n;                  // a power of two
        int es = (i1 * NS) & (n - 1);                 // i1 NS < n
        if (es >= n / 2) es -= n;
        C step[R];
        twiddle_powers<R, T>((T)(2 * SIGN) * (T)es * inv_n, step);
        int e0 = i1 * t;                              // < n
        if (e0 >= n / 2) e0 -= n;
        C w0 = expipi<T>((T)(2 * SIGN) * (T)e0 * inv_n);
        C rho = C{(T)1, (T)0};
        if constexpr (J > 1) {
            int er = i1 * (L / 16);                   // < n / 16
            if (er >= n / 2) er -= n;
            rho = expipi<T>((T)(2 * SIGN) * (T)er * inv_n);
        }
#pragma unroll
        for (int jb = 0; jb < J; ++jb) {
            const int jj = t + jb * (L / 16);
            if (jb > 0) w0 = cmul(w0, rho);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int l2 = jj + r * NS;
                out[(int64_t)l2 * n1 + i1] = cmul(v[jb * R + r], cmul(w0, step[r]));
            }
        }
    }
}

// acc += w g[off] for a row of the fused gather (off < 0: no such row).
template <typename C> __device__ __forceinline__ void fused_tap(float2& acc, float w, const C* col, int off) {
    if (off < 0) return;
    const C g = col[off];
    acc.x += w * g.x;
    acc.y += w * g.y;
}

// Pass 2 for a tile of TILES rows l2: the length-n1 FFTs over i1 of
// Y[l2 n1 + i1], stored to X[l2 + n2 l1] (natural order of the length-n
// transform) in the band grid.  For float rows of 2^(4j+3) points the first
// stage is radix 8 with two butterflies per thread, so each thread reads 8
// pairs of adjacent elements with 16-byte loads.
//
// Fused gather (FP32 forward, bands with B.fused): the grid is not stored.
// The tile's rows stay in shared memory in natural order, and every entry of
// the tile's row block -- one node and the taps of its window that fall in
// these rows, all at one column l1 -- sums phi_rho g[rho][l1] over the rows
// into its slot of the band's partial sums; the gather kernel adds a node's
// slots and recombines the right-hand sides.
template <typename T, int SIGN, int LOG2L>
__global__ void __launch_bounds__(PassTile<T, LOG2L, PassBudget<T>::P2>::NT,
                                  PassTile<T, LOG2L, PassBudget<T>::P2>::MINB)
    k_pass2(const PassItem* __restrict__ items, const BandDev* __restrict__ bands, int log2n2,
            const C_t<T>* __restrict__ Y, C_t<T>* __restrict__ dst, const C_t<T>* __restrict__ tw,
            FuseArgs fz) {
    using C = C_t<T>;
    using PT = PassTile<T, LOG2L, PassBudget<T>::P2>;
    constexpr int L = PT::L, TR = PT::TILES, LD = PT::LD;
    constexpr int FIRST = (sizeof(T) == 4 && LOG2L % 4 == 3) ? 3 : 4;
    extern __shared__ unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const PassItem item = items[blockIdx.y];
    const BandDev B = bands[item.band];
    const int n = L << log2n2;
    const int s = item.rhs;
    const int l2b = blockIdx.x * TR;
    const int tid = threadIdx.x;
    const C* in = Y + item.y_off + (int64_t)l2b * L;
    const C* twr = tw + tw_region(LOG2L, FIRST);
    // first stage straight from the rows (consecutive threads, consecutive i1)
    {
        const int row = tid / (L / 16), t = tid & (L / 16 - 1);
        C v[16];
        C* buf = sm + row * LD;
        if constexpr (FIRST == 3) {
            // pair t + r L/16 holds elements 2t + r L/8 and 2t + 1 + r L/8
            const float4* in4 = reinterpret_cast<const float4*>(in + (int64_t)row * L);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float4 q2 = in4[t + r * (L / 16)];
                v[r] = C{q2.x, q2.y};
                v[8 + r] = C{q2.z, q2.w};
            }
            fft_first8x2_from_regs<LOG2L, SIGN, T>(v, buf, t);
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = in[(int64_t)row * L + t + r * (L / 16)];
            fft_first_from_regs<LOG2L, SIGN, T>(v, buf, t);
        }
        fft_middle<LOG2L, FIRST, SIGN, T>(buf, t, twr);
    }
    // last stage with rows fastest: the warp's stores are TR-row segments of X
    {
        using SP = StagePlan<LOG2L, FIRST>;
        constexpr int R = SP::LAST_R, NS = SP::LAST_NS, J = 16 / R;
        const int row = tid & (TR - 1), t = tid >> PT::LOG2T;
        C v[16];
        fft_last_to_regs<LOG2L, FIRST, SIGN, T>(sm + row * LD, t, v, twr);
        if constexpr (sizeof(T) == 4 && SIGN > 0) {
            if (B.fused) {
                __syncthreads();   // every thread has read its last-stage inputs
                C* rbuf = sm + row * LD;
#pragma unroll
                for (int jb = 0; jb < J; ++jb) {
                    const int jj = t + jb * (L / 16);
#pragma unroll
                    for (int r = 0; r < R; ++r) rbuf[jj + r * NS] = v[jb * R + r];
                }
                __syncthreads();
                // entries of this row block: [e0, e1) of the band's list
                const int e0 = fz.rbs[B.rbs_off + blockIdx.x], e1 = fz.rbs[B.rbs_off + blockIdx.x + 1];
                constexpr int NQ = (TR + 3) / 4;   // float4 of window values per entry
                const int2* ent = fz.ent + B.ent_off;
                const float4* ph = fz.phi + B.ph_off;
                float2* pp = fz.pp + B.pp_off + (int64_t)s * B.nodes * B.pparts;
                for (int e = e0 + tid; e < e1; e += PT::NT) {
                    const int2 a = __ldg(ent + e);
                    const C* col = sm + a.y;
                    float2 acc = {0.f, 0.f};
#pragma unroll
                    for (int qd = 0; qd < NQ; ++qd) {
                        const float4 w4 = __ldg(ph + e * NQ + qd);
                        fused_tap(acc, w4.x, col, 4 * qd + 0 < TR ? (4 * qd + 0) * LD : -1);
                        fused_tap(acc, w4.y, col, 4 * qd + 1 < TR ? (4 * qd + 1) * LD : -1);
                        fused_tap(acc, w4.z, col, 4 * qd + 2 < TR ? (4 * qd + 2) * LD : -1);
                        fused_tap(acc, w4.w, col, 4 * qd + 3 < TR ? (4 * qd + 3) * LD : -1);
                    }
                    pp[a.x] = acc;
                }
                return;
            }
        }
        C* out = dst + B.grid_off + (int64_t)s * n + l2b + row;
#pragma unroll
        for (int jb = 0; jb < J; ++jb) {
            const int jj = t + jb * (L / 16);
#pragma unroll
            for (int r = 0; r < R; ++r) out[(int64_t)(jj + r * NS) << log2n2] = v[jb * R + r];
        }
    }
}


// The smallest shared-memory carveout that still holds `ctas` CTAs of `smem`
// bytes (plus the 1 KiB each reserves) in the SM's 228 KiB, so that the rest
// stays L1 for the stage-twiddle table and the passes' input loads: measured
// at N = M = 2^20 FP32, both passes 15 % faster than with the whole storage
// as shared memory.
static inline int pass_carveout(size_t smem, int ctas) {
    if (FL_PASS_CARVEOUT >= 0) return FL_PASS_CARVEOUT;
    const double need = (double)ctas * (double)(smem + 1024);
    const int pct = (int)ceil(100.0 * need / (228.0 * 1024.0)) + 1;
    return pct < 0 ? 0 : (pct > 100 ? 100 : pct);
}

// Host launchers: one launch covers the work items items[0..nitems) (one per
// (band, right-hand side) of one grid size); the pass length picks the compiled
// instantiation.

template <typename T, int SIGN, int MODE, bool DERIV, int LOG2L>
static cudaError_t pass1_ct(const PassItem* items, int nitems, const BandDev* bands, int log2n1,
                            const C_t<T>* c, const T* D, const C_t<T>* src, C_t<T>* Y,
                            const C_t<T>* tw, cudaStream_t st) {
    using PT = PassTile<T, LOG2L, PassBudget<T>::P1, FL_P1_SEG_BYTES>;
    auto k = k_pass1<T, SIGN, MODE, DERIV, LOG2L>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PT::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 pass_carveout(PT::SMEM, PT::MINB));
    if (e != cudaSuccess) return e;
    k<<<dim3((unsigned)((1 << log2n1) / PT::TILES), (unsigned)nitems), PT::NT, PT::SMEM, st>>>(
        items, bands, log2n1, c, D, src, Y, tw);
    return cudaGetLastError();
}

template <typename T, int SIGN, int LOG2L>
static cudaError_t pass2_ct(const PassItem* items, int nitems, const BandDev* bands, int log2n2,
                            const C_t<T>* Y, C_t<T>* dst, const C_t<T>* tw, FuseArgs fz,
                            cudaStream_t st) {
    using PT = PassTile<T, LOG2L, PassBudget<T>::P2>;
    auto k = k_pass2<T, SIGN, LOG2L>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PT::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 pass_carveout(PT::SMEM, PT::MINB));
    if (e != cudaSuccess) return e;
    k<<<dim3((unsigned)((1 << log2n2) / PT::TILES), (unsigned)nitems), PT::NT, PT::SMEM, st>>>(
        items, bands, log2n2, Y, dst, tw, fz);
    return cudaGetLastError();
}

// Pass 1 (length n2 = 2^log2n2, 6..12) over all n1 = 2^log2n1 columns.
template <typename T, int SIGN, int MODE, bool DERIV>
cudaError_t launch_pass1(const PassItem* items, int nitems, const BandDev* bands, int log2n1,
                         int log2n2, const C_t<T>* c, const T* D, const C_t<T>* src, C_t<T>* Y,
                         const C_t<T>* tw, cudaStream_t st) {
    switch (log2n2) {
#define FL_P1(LG) \
    case LG: return pass1_ct<T, SIGN, MODE, DERIV, LG>(items, nitems, bands, log2n1, c, D, src, Y, tw, st);
        FL_P1(6) FL_P1(7) FL_P1(8) FL_P1(9) FL_P1(10) FL_P1(11) FL_P1(12)
#undef FL_P1
        default: return cudaErrorInvalidValue;
    }
}

// Pass 2 (length n1 = 2^log2n1, 7..12) over all n2 = 2^log2n2 rows.
template <typename T, int SIGN>
cudaError_t launch_pass2(const PassItem* items, int nitems, const BandDev* bands, int log2n1,
                         int log2n2, const C_t<T>* Y, C_t<T>* dst, const C_t<T>* tw, FuseArgs fz,
                         cudaStream_t st) {
    switch (log2n1) {
#define FL_P2(LG) \
    case LG: return pass2_ct<T, SIGN, LG>(items, nitems, bands, log2n2, Y, dst, tw, fz, st);
        FL_P2(6) FL_P2(7) FL_P2(8) FL_P2(9) FL_P2(10) FL_P2(11) FL_P2(12)
#undef FL_P2
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// FFTs of the grids of at most 4096 points: one CTA of 256 threads per work
// item (nfft FFTs of one band, nfft n <= 4096).  n >= 64: the compile-time
// radix-16 transform above with 16 points per thread and the plan-time stage
// twiddles; n = 32: the generic radix-8 transform of fl_common.cuh (8 points
// per thread).  MODE 0: input generated from c and D (forward), written to the
// band grid; MODE 1: the grid read and transformed in place.
constexpr int kSmallThreads = 256;

template <typename T, int SIGN, int MODE, bool DERIV, int LOG2L>
__device__ __forceinline__ void small_fft_ct(const SmallWork& wk, const BandDev& B,
                                             const C_t<T>* __restrict__ c, const T* __restrict__ D,
                                             C_t<T>* __restrict__ grid, const C_t<T>* __restrict__ tw,
                                             C_t<T>* sm) {
    using C = C_t<T>;
    using SP = StagePlan<LOG2L>;
    constexpr int L = 1 << LOG2L, NT = L / 16;
    const int f = threadIdx.x / NT, t = threadIdx.x % NT;   // f < 4096 / L: own smem region
    const bool active = f < wk.nfft;
    const int s = wk.s0 + f;
    C* g = grid + B.grid_off + (int64_t)s * L;
    C v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int e = t + r * (L / 16);
        v[r] = !active ? C{(T)0, (T)0}
                       : (MODE == 0 ? prep_value<T, DERIV>(e, B, s, c + B.c_off, D) : g[e]);
    }
    C* buf = sm + f * L;
    const C* twr = tw + tw_region(LOG2L, 4);
    fft_first_from_regs<LOG2L, SIGN, T>(v, buf, t);
    fft_middle<LOG2L, 4, SIGN, T>(buf, t, twr);
    fft_last_to_regs<LOG2L, 4, SIGN, T>(buf, t, v, twr);
    if (!active) return;
    constexpr int R = SP::LAST_R, NS = SP::LAST_NS, J = 16 / R;
#pragma unroll
    for (int jb = 0; jb < J; ++jb) {
        const int jj = t + jb * (L / 16);
#pragma unroll
        for (int r = 0; r < R; ++r) g[jj + r * NS] = v[jb * R + r];
    }
}

template <typename T, int SIGN, int MODE, bool DERIV>
__global__ void __launch_bounds__(kSmallThreads) k_small_fft(const SmallWork* __restrict__ work,
                                                             const BandDev* __restrict__ bands,
                                                             const C_t<T>* __restrict__ c,
                                                             const T* __restrict__ D,
                                                             C_t<T>* __restrict__ grid,
                                                             const C_t<T>* __restrict__ tw) {
    using C = C_t<T>;
    extern __shared__ unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const SmallWork wk = work[blockIdx.x];
    const BandDev B = bands[wk.band];
    switch (wk.log2n) {
#define FL_SMALL(LG) \
    case LG: small_fft_ct<T, SIGN, MODE, DERIV, LG>(wk, B, c, D, grid, tw, sm); return;
        FL_SMALL(6) FL_SMALL(7) FL_SMALL(8) FL_SMALL(9) FL_SMALL(10) FL_SMALL(11) FL_SMALL(12)
#undef FL_SMALL
        default: break;
    }
    // n = 32 (at most 64 FFTs per item): radix 8 with per-stage twiddles
    const int L = 1 << wk.log2n;
    const int nthr = L >> 3;
    const int f = threadIdx.x / nthr, t = threadIdx.x % nthr;
    const bool active = f < wk.nfft;
    const int s = wk.s0 + f;
    C* buf = sm + (int64_t)f * padded_len(L);
    C* g = grid + B.grid_off + (int64_t)s * L;
    if (active) {
        for (int e = t; e < L; e += nthr)
            buf[pad8(e)] = (MODE == 0) ? prep_value<T, DERIV>(e, B, s, c + B.c_off, D) : g[e];
    }
    __syncthreads();
    fft_smem<SIGN, T>(buf, wk.log2n, t, active);
    if (active)
        for (int e = t; e < L; e += nthr) g[e] = buf[pad8(e)];
}

// The same work items with 512 threads, 8 points per thread and the generic
// radix-8 transform for every n: shorter per-thread chains, the faster choice
// when there are too few items to fill the GPU.
template <typename T, int SIGN, int MODE, bool DERIV>
__global__ void __launch_bounds__(2 * kSmallThreads) k_small_fft_r8(const SmallWork* __restrict__ work,
                                                                    const BandDev* __restrict__ bands,
                                                                    const C_t<T>* __restrict__ c,
                                                                    const T* __restrict__ D,
                                                                    C_t<T>* __restrict__ grid) {
    using C = C_t<T>;
    extern __shared__ unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const SmallWork wk = work[blockIdx.x];
    const BandDev B = bands[wk.band];
    const int L = 1 << wk.log2n;
    const int nthr = L >> 3;
    const int f = threadIdx.x / nthr, t = threadIdx.x % nthr;
    const bool active = f < wk.nfft;
    const int s = wk.s0 + f;
    C* buf = sm + (int64_t)f * padded_len(L);
    C* g = grid + B.grid_off + (int64_t)s * L;
    if (active) {
        for (int e = t; e < L; e += nthr)
            buf[pad8(e)] = (MODE == 0) ? prep_value<T, DERIV>(e, B, s, c + B.c_off, D) : g[e];
    }
    __syncthreads();
    fft_smem<SIGN, T>(buf, wk.log2n, t, active);
    if (active)
        for (int e = t; e < L; e += nthr) g[e] = buf[pad8(e)];
}

template <typename T, int SIGN, int MODE, bool DERIV>
cudaError_t launch_small_fft(const SmallWork* work, int nwork, const BandDev* bands, const C_t<T>* c,
                             const T* D, C_t<T>* grid, const C_t<T>* tw, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (nwork >= 2 * sms) {   // enough items: the radix-16 kernel
        const size_t smem = (size_t)4096 * sizeof(C_t<T>);
        auto k = k_small_fft<T, SIGN, MODE, DERIV>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)nwork, kSmallThreads, smem, st>>>(work, bands, c, D, grid, tw);
    } else {
        const size_t smem = (size_t)padded_len(4096) * sizeof(C_t<T>);
        auto k = k_small_fft_r8<T, SIGN, MODE, DERIV>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)nwork, 2 * kSmallThreads, smem, st>>>(work, bands, c, D, grid);
    }
    return cudaGetLastError();
}

#define FL_SMALL_SIG(T) const SmallWork*, int, const BandDev*, const C_t<T>*, const T*, C_t<T>*, \
                        const C_t<T>*, cudaStream_t

#define FL_P1_SIG(T) const PassItem*, int, const BandDev*, int, int, const C_t<T>*, const T*, \
                     const C_t<T>*, C_t<T>*, const C_t<T>*, cudaStream_t
#define FL_P2_SIG(T) const PassItem*, int, const BandDev*, int, int, const C_t<T>*, C_t<T>*, \
                     const C_t<T>*, FuseArgs, cudaStream_t
#define FL_FFT_EXTERN(T)                                                   \
    extern template cudaError_t launch_pass1<T, 1, 0, false>(FL_P1_SIG(T)); \
    extern template cudaError_t launch_pass1<T, 1, 0, true>(FL_P1_SIG(T));  \
    extern template cudaError_t launch_pass1<T, -1, 1, false>(FL_P1_SIG(T)); \
    extern template cudaError_t launch_pass1<T, 1, 1, false>(FL_P1_SIG(T));  \
    extern template cudaError_t launch_pass2<T, 1>(FL_P2_SIG(T));          \
    extern template cudaError_t launch_pass2<T, -1>(FL_P2_SIG(T));          \
    extern template cudaError_t launch_small_fft<T, 1, 0, false>(FL_SMALL_SIG(T)); \
    extern template cudaError_t launch_small_fft<T, 1, 0, true>(FL_SMALL_SIG(T));  \
    extern template cudaError_t launch_small_fft<T, -1, 1, false>(FL_SMALL_SIG(T)); \
    extern template cudaError_t launch_small_fft<T, 1, 1, false>(FL_SMALL_SIG(T));
// float pairs: the forward transform only
#define FL_FFT_EXTERN_FF                                                      \
    extern template cudaError_t launch_pass1<ff, 1, 0, false>(FL_P1_SIG(ff)); \
    extern template cudaError_t launch_pass2<ff, 1>(FL_P2_SIG(ff));           \
    extern template cudaError_t launch_small_fft<ff, 1, 0, false>(FL_SMALL_SIG(ff));

}  // namespace fl
