// fl_laplace.cu -- Algorithm 1 of Kunis & Melzer (Section 3): the real discrete
// Laplace transform f_j = sum_k c_k exp(-s_j t_k) through the hierarchical
// factorisation K~ = diag(L^{Y_m}) (K^{Y_m,Omega_l}) diag(L^{Omega_l})^T plus the
// cumulative sums g_m (Definition 3.2, Theorem A.3):
//
//   g_M = sum_{t_k in Omega_M} c_k,  g_m = g_{m+1} + sum_{t_k in Omega_m} c_k
//   v^{Omega_l}_r = sum_{t_k in Omega_l} L_r^{Omega_l}(t_k) c_k         (moments)
//   h^{Y_m}_s = sum_{l=l_m}^{L_m} sum_r K^{Y_m,Omega_l}_{s r} v^{Omega_l}_r (coupling)
//   f~_j = sum_s L_s^{Y_m}(s_j) h^{Y_m}_s + g_{L_m+1}  (s_j in Y_m),  g_1 (s_j in Y_M)
//
// Kernels: k_lap_minmax (interval ends y_1 = max s, xi_1 = max t, validity),
// k_lap_band (band of every t_k and s_j), k_lap_moments (moments and band sums,
// deterministic: per-warp tables, warp-ordered group sums, block partials
// reduced in block order by k_lap_reduce), k_lap_couple (h and g), k_lap_eval.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "fl_plan.cuh"

namespace fl {

constexpr int kLapWarps = 8;          // warps per moment block
constexpr int kLapMaxBlocks = 128;    // moment blocks (fixed: partial-sum order)

__device__ __forceinline__ int lap_band(double v, double v1, int levels) {
    if (levels <= 1) return 1;
    if (v > ldexp(v1, -1)) return 1;
    if (!(v > ldexp(v1, -(levels - 1)))) return levels;
    int b = (int)floor(log2(v1 / v)) + 1;
    b = max(1, min(b, levels - 1));
    while (b > 1 && v > ldexp(v1, -(b - 1))) --b;
    while (b < levels - 1 && !(v > ldexp(v1, -b))) ++b;
    return b;
}

// max over non-negative doubles by their bit patterns (monotone for x >= 0);
// flag bit 1: a t_k or s_j is negative or not finite.
__global__ void k_lap_minmax(int64_t N, const double* __restrict__ t, int64_t M,
                             const double* __restrict__ s, unsigned long long* __restrict__ mx,
                             int* __restrict__ flag) {
    unsigned long long mt = 0, ms = 0;
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const double v = t[i];
        if (!(v >= 0.0) || !isfinite(v)) bad = 1;
        else mt = max(mt, (unsigned long long)__double_as_longlong(v));
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const double v = s[i];
        if (!(v >= 0.0) || !isfinite(v)) bad = 1;
        else ms = max(ms, (unsigned long long)__double_as_longlong(v));
    }
    if (bad) atomicOr(flag, 1);
    atomicMax(&mx[0], mt);
    atomicMax(&mx[1], ms);
}

__global__ void k_lap_band(int64_t n, const double* __restrict__ v, double v1, int levels,
                           uint8_t* __restrict__ band) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) band[i] = (uint8_t)lap_band(v[i], v1, levels);
}

// Moments and band sums.  Table row l (1..levels) holds v^{Omega_l}_0..q-1 and,
// in column q, the band sum sum_{t_k in Omega_l} c_k.  Each warp owns a table;
// for every 32 consecutive t_k it takes, lanes are grouped by band
// (match_any) and each group's sum is formed in lane order and added by the
// group's lowest lane, so the result does not depend on scheduling.
template <typename T, bool BANDS_FROM_VALUES = false>
__global__ void k_lap_moments(int64_t N, const double* __restrict__ t,
                              const uint8_t* __restrict__ tband, const T* __restrict__ c,
                              int levels, int q, double xi1, const double* __restrict__ cheb,
                              T* __restrict__ partial) {
    extern __shared__ unsigned char smem_raw[];
    T* tab = reinterpret_cast<T*>(smem_raw);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;   // warps (tables) per block
    const int row = q + 1;
    const int entries = (levels + 1) * row;
    for (int i = threadIdx.x; i < nw * entries; i += blockDim.x) tab[i] = (T)0;
    __syncthreads();
    T* mytab = tab + w * entries;
    const int64_t nchunk = (N + 31) / 32;
    for (int64_t ch = (int64_t)blockIdx.x * nw + w; ch < nchunk; ch += (int64_t)gridDim.x * nw) {
        const int64_t k = ch * 32 + lane;
        const bool valid = k < N;
        const int l = !valid ? 255 : (BANDS_FROM_VALUES ? lap_band(t[k], xi1, levels) : tband[k]);
        const double cv = valid ? (double)c[k] : 0.0;
        // barycentric denominator on Omega_l (only for interpolated bands)
        double tau = 0.0, inv_den = 1.0;
        int hit = -1;
        const bool interp = valid && l < levels;
        if (interp) {
            const double a = ldexp(xi1, -l);
            tau = (t[k] - 1.5 * a) / (0.5 * a);
            double den = 0.0;
            for (int r = 0; r < q; ++r) {
                const double d = tau - cheb[r];
                if (d == 0.0) hit = r;
                den += cheb[q + r] / d;
            }
            inv_den = 1.0 / den;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, l);
        const bool leader = (peers & ((1u << lane) - 1u)) == 0u;
        for (int r = 0; r <= q; ++r) {
            T val = (T)0;
            if (r == q) {
                val = (T)cv;
            } else if (interp) {
                const double Lr = (hit >= 0) ? (r == hit ? 1.0 : 0.0)
                                             : (cheb[q + r] / (tau - cheb[r])) * inv_den;
                val = (T)(Lr * cv);
            }
            T acc = (T)0;
            for (int src = 0; src < 32; ++src) {
                const T x = __shfl_sync(0xffffffffu, val, src);
                if ((peers >> src) & 1u) acc += x;
            }
            if (valid && leader) mytab[l * row + r] += acc;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < entries; i += blockDim.x) {
        T s = (T)0;
        for (int ww = 0; ww < nw; ++ww) s += tab[ww * entries + i];
        partial[(int64_t)blockIdx.x * entries + i] = s;
    }
}

// Largest rank any Laplace plan uses (Algorithm 1: kMaxQ; the generalised
// algorithm: kGenMaxQ below): the size of the per-element weight arrays.
constexpr int kLapMaxRank = 64;

// Barycentric weights w_r = lambda_r / (tau - t_r), r < q, with one division:
// Montgomery's batch inversion (prefix products of d_r = tau - t_r, one
// reciprocal, a backward sweep), about 3q ulps instead of 1/2 ulp per weight.
// Returns false and leaves hit = r when some d_r is exactly zero.
__device__ __forceinline__ bool bary_batch(double tau, int q, const double* __restrict__ cheb,
                                           double* w, int* hit) {
    double pre = 1.0;
    for (int r = 0; r < q; ++r) {
        const double d = tau - cheb[r];
        if (d == 0.0) {
            *hit = r;
            return false;
        }
        w[r] = pre;                      // product of d_0 .. d_{r-1}
        pre *= d;
    }
    double inv = 1.0 / pre;              // 1 / (d_0 ... d_{q-1})
    for (int r = q - 1; r >= 0; --r) {
        const double d = tau - cheb[r];
        const double ir = inv * w[r];    // 1 / d_r
        inv *= d;
        w[r] = cheb[q + r] * ir;
    }
    return true;
}

// The moments of k_lap_moments for t_k in band order (plan time, a stable
// sort by band): t, tband sorted, c read through tperm.  A warp's 32 elements
// then form runs of equal band, so each moment is summed per run by a
// segmented shuffle scan (5 steps instead of 32) whose last lane adds it to
// the warp's table; the runs of one chunk have distinct bands, so no two lanes
// add to one entry and the order stays fixed.  Each weight lambda_r / (tau - t_r)
// is formed once.
template <typename T>
__global__ void k_lap_moments_sorted(int64_t N, const double* __restrict__ t,
                                     const uint8_t* __restrict__ tband,
                                     const int32_t* __restrict__ tperm, const T* __restrict__ c,
                                     int levels, int q, double xi1, const double* __restrict__ cheb,
                                     T* __restrict__ partial) {
    extern __shared__ unsigned char smem_raw[];
    T* tab = reinterpret_cast<T*>(smem_raw);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int row = q + 1;
    const int entries = (levels + 1) * row;
    for (int i = threadIdx.x; i < nw * entries; i += blockDim.x) tab[i] = (T)0;
    __syncthreads();
    T* mytab = tab + w * entries;
    const int64_t nchunk = (N + 31) / 32;
    for (int64_t ch = (int64_t)blockIdx.x * nw + w; ch < nchunk; ch += (int64_t)gridDim.x * nw) {
        const int64_t k = ch * 32 + lane;
        const bool valid = k < N;
        const int l = valid ? tband[k] : 255;       // invalid lanes: a run of their own at the end
        const double cv = valid ? (double)c[tperm[k]] : 0.0;
        double tau = 0.0, inv_den = 1.0;
        double wr[kLapMaxRank];
        int hit = -1;
        const bool interp = valid && l < levels;
        if (interp) {
            const double a = ldexp(xi1, -l);
            tau = (t[k] - 1.5 * a) / (0.5 * a);
            if (bary_batch(tau, q, cheb, wr, &hit)) {
                double den = 0.0;
                for (int r = 0; r < q; ++r) den += wr[r];
                inv_den = 1.0 / den;
            }
        }
        // runs of equal band: s0 = first lane of my run, tail = last lane of it
        const int lprev = __shfl_up_sync(0xffffffffu, l, 1);
        const bool head = lane == 0 || lprev != l;
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        const int s0 = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
        for (int r = 0; r <= q; ++r) {
            T val = (T)0;
            if (r == q) {
                val = (T)cv;
            } else if (interp) {
                const double Lr = (hit >= 0) ? (r == hit ? 1.0 : 0.0) : wr[r] * inv_den;
                val = (T)(Lr * cv);
            }
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const T x = __shfl_up_sync(0xffffffffu, val, off);
                if (lane - off >= s0) val += x;
            }
            if (valid && tail) mytab[l * row + r] += val;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < entries; i += blockDim.x) {
        T s = (T)0;
        for (int ww = 0; ww < nw; ++ww) s += tab[ww * entries + i];
        partial[(int64_t)blockIdx.x * entries + i] = s;
    }
}

// vS[i] = sum over blocks of partial[b][i]: one warp per entry, lane l summing
// the blocks l, l + 32, ... and a fixed shuffle tree combining the lanes.
template <typename T>
__global__ void k_lap_reduce(int nblocks, int entries, const T* __restrict__ partial,
                             double* __restrict__ vS) {
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= entries) return;                    // uniform across the warp
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += (double)partial[(int64_t)b * entries + i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) vS[i] = s;
}

// h^{Y_m}_s for m = blockIdx.x + 1 (threads over s) with
// K^{Y_m,Omega_l}_{s r} = exp(-y_s xi_r) formed on the fly; block 0 also forms
// the cumulative sums g_l = sum_{l' >= l} S_{l'}, g_{levels+1} = 0.
__global__ void k_lap_couple(int levels, int q, double y1, double xi1,
                             const int* __restrict__ ell, const double* __restrict__ cheb,
                             const double* __restrict__ vS, double* __restrict__ h,
                             double* __restrict__ g) {
    const int m = blockIdx.x + 1;
    const int row = q + 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        g[levels + 1] = 0.0;
        for (int l = levels; l >= 1; --l) g[l] = g[l + 1] + vS[l * row + q];
    }
    if (m >= levels) return;
    const int s = threadIdx.x;
    if (s >= q) return;
    const double ay = ldexp(y1, -m);
    const double ys = 1.5 * ay + 0.5 * ay * cheb[s];
    double acc = 0.0;
    for (int l = ell[m]; l <= levels - m; ++l) {
        const double ax = ldexp(xi1, -l);
        for (int r = 0; r < q; ++r) {
            const double xr = 1.5 * ax + 0.5 * ax * cheb[r];
            acc += exp(-ys * xr) * vS[l * row + r];
        }
    }
    h[m * q + s] = acc;
}

// Plan-time table of the coupling blocks: Kt[koff[m] + ((l - l_m) q + s) q + r]
// = exp(-y_s^{Y_m} xi_r^{Omega_l}), the same expression k_lap_couple evaluates.
__global__ void k_lap_ktable(int levels, int q, double y1, double xi1, const int* __restrict__ ell,
                             const int64_t* __restrict__ koff, const double* __restrict__ cheb,
                             double* __restrict__ Kt) {
    const int m = blockIdx.x + 1;
    if (m >= levels) return;
    const int nl = levels - m - ell[m] + 1;
    const double ay = ldexp(y1, -m);
    for (int i = threadIdx.x; i < nl * q * q; i += blockDim.x) {
        const int r = i % q, s = (i / q) % q, l = ell[m] + i / (q * q);
        const double ys = 1.5 * ay + 0.5 * ay * cheb[s];
        const double ax = ldexp(xi1, -l);
        const double xr = 1.5 * ax + 0.5 * ax * cheb[r];
        Kt[koff[m] + i] = exp(-ys * xr);
    }
}

// k_lap_couple with the coupling blocks read from the plan's table (same
// summation order, so the same h).
__global__ void k_lap_couple_tab(int levels, int q, const int* __restrict__ ell,
                                 const int64_t* __restrict__ koff, const double* __restrict__ Kt,
                                 const double* __restrict__ vS, double* __restrict__ h,
                                 double* __restrict__ g) {
    const int m = blockIdx.x + 1;
    const int row = q + 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        g[levels + 1] = 0.0;
        for (int l = levels; l >= 1; --l) g[l] = g[l + 1] + vS[l * row + q];
    }
    if (m >= levels) return;
    // one warp per s: lanes stride over the (l, r) terms, a fixed shuffle tree
    // combines them
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int l0 = ell[m];
    const int tot = max(levels - m - l0 + 1, 0) * q;
    const double* K = Kt + koff[m];
    for (int s = warp; s < q; s += nw) {
        double acc = 0.0;
        for (int i = lane; i < tot; i += 32) {
            const int li = i / q, r = i - li * q;
            acc += K[((int64_t)li * q + s) * q + r] * vS[(l0 + li) * row + r];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) h[m * q + s] = acc;
    }
}

// f~_j: barycentric weights of s_j on Y_m (double), then sum_s L_s h_s + g_{L_m + 1}.
template <typename T, bool BANDS_FROM_VALUES = false>
__global__ void k_lap_eval(int64_t M, const double* __restrict__ sv,
                           const uint8_t* __restrict__ sband, int levels, int q, double y1,
                           const double* __restrict__ cheb, const double* __restrict__ h,
                           const double* __restrict__ g, T* __restrict__ f) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int m = BANDS_FROM_VALUES ? lap_band(sv[j], y1, levels) : sband[j];
    if (m >= levels) {
        f[j] = (T)g[1];
        return;
    }
    const double a = ldexp(y1, -m);
    const double tau = (sv[j] - 1.5 * a) / (0.5 * a);
    double w[kMaxQ];
    int hit = -1;
    double interp;
    if (bary_batch(tau, q, cheb, w, &hit)) {
        double den = 0.0, num = 0.0;
        for (int s = 0; s < q; ++s) {
            den += w[s];
            num += w[s] * h[m * q + s];
        }
        interp = num / den;
    } else {
        interp = h[m * q + hit];
    }
    f[j] = (T)(interp + g[levels - m + 1]);
}

// Chebyshev points and barycentric weights (Section 2); same table as Algorithm 2.
__global__ void k_lap_cheb(int q, double* cheb) {
    const int s = threadIdx.x;
    if (s >= q) return;
    double sn, cs;
    sincospi((2.0 * s + 1.0) / (2.0 * q), &sn, &cs);
    cheb[s] = cs;
    cheb[q + s] = (s & 1) ? -sn : sn;
}

// ---------------------------------------------------------------------------
// Generalised Algorithm 1 (Section 3, the theorem after Algorithm 1): an
// asymptotically smooth kernel kappa(y, xi) in place of exp(-y xi).  Every
// block Y_m x Omega_l with 1 <= m, l <= M - 1 is interpolated (no block is
// replaced by 0 or 1), the near fields Y_M (every frequency) and Omega_M (every
// node) are summed directly, and M = ceil(log2(y_1 xi_1 N / eps)) + 1.
// Kernels: kind 1 exp(-y xi); kind 2 K_{1/2}(y xi) = sqrt(pi / (2 y xi)) exp(-y xi)
// (the example there, y, xi > 0).

constexpr int kGenMaxQ = 64;
static_assert(kGenMaxQ <= kLapMaxRank && kMaxQ <= kLapMaxRank, "weight arrays of the moments kernel");

__device__ __forceinline__ double gen_kappa(int kind, double y, double xi) {
    const double x = y * xi;
    return kind == 2 ? sqrt(1.5707963267948966192313216916398 / x) * exp(-x) : exp(-x);
}

// Kt[((m - 1)(M - 1) + l - 1) q^2 + s q + r] = kappa(y_s^{Y_m}, xi_r^{Omega_l}), block m.
__global__ void k_gen_ktable(int kind, int levels, int q, double y1, double xi1,
                             const double* __restrict__ cheb, double* __restrict__ Kt) {
    const int m = blockIdx.x + 1;
    const int nb = levels - 1;
    const double ay = ldexp(y1, -m);
    for (int i = threadIdx.x; i < nb * q * q; i += blockDim.x) {
        const int r = i % q, s = (i / q) % q, l = 1 + i / (q * q);
        const double ys = 1.5 * ay + 0.5 * ay * cheb[s];
        const double ax = ldexp(xi1, -l);
        const double xr = 1.5 * ax + 0.5 * ax * cheb[r];
        Kt[(int64_t)(m - 1) * nb * q * q + i] = gen_kappa(kind, ys, xr);
    }
}

// h^{Y_m}_s = sum_{l = 1}^{M - 1} sum_r Kt(m, l)_{s r} v^{Omega_l}_r, m = blockIdx.x + 1.
// One warp per s: lanes stride over the (l, r) terms, a fixed shuffle tree
// combines them.
__global__ void k_gen_couple(int levels, int q, const double* __restrict__ Kt,
                             const double* __restrict__ vS, double* __restrict__ h) {
    const int m = blockIdx.x + 1, row = q + 1, nb = levels - 1;
    if (m >= levels) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int tot = nb * q;
    for (int s = warp; s < q; s += nw) {
        double acc = 0.0;
        for (int i = lane; i < tot; i += 32) {
            const int li = i / q, r = i - li * q;      // l = li + 1
            acc += Kt[(((int64_t)(m - 1) * nb + li) * q + s) * q + r] * vS[(li + 1) * row + r];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) h[m * q + s] = acc;
    }
}

// f~_j: s_j in Y_m (m < M): sum_s L_s^{Y_m}(s_j) h^{Y_m}_s plus the Omega_M near
// field sum_{t_k in Omega_M} c_k kappa(s_j, t_k); s_j in Y_M: the direct sum.
template <typename T, int KIND>
__global__ void k_gen_eval(int64_t M, const double* __restrict__ sv,
                           const uint8_t* __restrict__ sband, int levels, int q, double y1,
                           const double* __restrict__ cheb, const double* __restrict__ h, int64_t N,
                           const double* __restrict__ t, const T* __restrict__ c,
                           const int32_t* __restrict__ nearT, int64_t nnear, T* __restrict__ f) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int m = sband[j];
    const double sj = sv[j];
    double acc = 0.0;
    if (m >= levels) {
        for (int64_t k = 0; k < N; ++k) acc += (double)c[k] * gen_kappa(KIND, sj, t[k]);
    } else {
        const double a = ldexp(y1, -m);
        const double tau = (sj - 1.5 * a) / (0.5 * a);
        double den = 0.0, num = 0.0;
        int hit = -1;
        for (int s = 0; s < q; ++s) {
            const double d = tau - cheb[s];
            if (d == 0.0) hit = s;
            const double wgt = cheb[q + s] / d;
            den += wgt;
            num += wgt * h[m * q + s];
        }
        acc = (hit >= 0) ? h[m * q + hit] : num / den;
        for (int64_t i = 0; i < nnear; ++i) {
            const int32_t k = nearT[i];
            acc += (double)c[k] * gen_kappa(KIND, sj, t[k]);
        }
    }
    f[j] = (T)acc;
}

// flag bit 1: a t_k or s_j is zero (kind 2 is singular at y xi = 0)
__global__ void k_gen_positive(int64_t N, const double* __restrict__ t, int64_t M,
                               const double* __restrict__ s, int* __restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        if (!(t[i] > 0.0)) bad = 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride)
        if (!(s[i] > 0.0)) bad = 1;
    if (bad) atomicOr(flag, 1);
}

// ---------------------------------------------------------------------------
// Scratch layout of one Laplace evaluation (all offsets in bytes, 256-aligned).
struct LapLayout {
    size_t partial, vS, h, g, ell, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static LapLayout lap_layout(int levels, int q, int nblocks, size_t tsize) {
    LapLayout L;
    const size_t entries = (size_t)(levels + 1) * (q + 1);
    size_t off = 0;
    L.partial = off; off = align256(off + (size_t)nblocks * entries * tsize);
    L.vS = off;      off = align256(off + entries * sizeof(double));
    L.h = off;       off = align256(off + (size_t)(levels + 1) * q * sizeof(double));
    L.g = off;       off = align256(off + (size_t)(levels + 2) * sizeof(double));
    L.ell = off;     off = align256(off + (size_t)(levels + 1) * sizeof(int));
    L.total = off;
    return L;
}

static int lap_blocks(int64_t N) {
    const int64_t chunks = (N + 31) / 32;
    return (int)std::max<int64_t>(1, std::min<int64_t>(kLapMaxBlocks, (chunks + kLapWarps - 1) / kLapWarps));
}

// Parameters of Definition 3.2 for the whole eps (Algorithm 1).
struct LapParams {
    int q, levels;
    double y1, xi1;
    int ell[FL_MAX_LEVELS];
};

static bool lap_params(double eps, int q_in, double y1, double xi1, LapParams* P) {
    P->q = q_in > 0 ? q_in : (int)ceil(0.5 + log(1.0 / eps) / log(4.0));
    P->y1 = y1;
    P->xi1 = xi1;
    if (!(y1 > 0.0) || !(xi1 > 0.0)) {
        P->levels = 1;
    } else {
        P->levels = (int)std::max(1.0, ceil(log2(y1 * xi1 / eps)) + 1.0);
    }
    if (P->levels > 127 || P->q > kMaxQ) return false;
    for (int m = 0; m < FL_MAX_LEVELS; ++m) P->ell[m] = 0;
    for (int m = 1; m < P->levels; ++m) {
        const double lg = log2(y1 * xi1) - m - log2(log(1.0 / eps));
        P->ell[m] = std::max(1, (int)floor(lg) + 1);
    }
    return true;
}

// Launches moments -> reduce -> couple -> eval on `scratch` (layout above),
// with nblocks moment blocks; the layout reserves partial sums for
// layout_blocks >= nblocks blocks (0: nblocks).
template <typename T, bool BANDS_FROM_VALUES = false>
static cudaError_t lap_run(int64_t N, int64_t M, const double* t, const double* s,
                           const uint8_t* tband, const uint8_t* sband, const LapParams& P,
                           const double* cheb, const T* c, T* f, unsigned char* scratch,
                           int nblocks, cudaStream_t st, Plan* timed,
                           const double* Kt = nullptr, const int64_t* koff = nullptr,
                           const int32_t* tperm = nullptr, int layout_blocks = 0) {
    const LapLayout L = lap_layout(P.levels, P.q, std::max(nblocks, layout_blocks), sizeof(T));
    const int entries = (P.levels + 1) * (P.q + 1);
    T* partial = (T*)(scratch + L.partial);
    double* vS = (double*)(scratch + L.vS);
    double* h = (double*)(scratch + L.h);
    double* g = (double*)(scratch + L.g);
    const int* ell = (const int*)(scratch + L.ell);
    const size_t smem = (size_t)kLapWarps * entries * sizeof(T);
    int slot = -1;
    if (N > 0) {
        auto kern = k_lap_moments<T, BANDS_FROM_VALUES>;
        cudaError_t e = tperm ? cudaFuncSetAttribute(k_lap_moments_sorted<T>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                              : cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem);
        if (e != cudaSuccess) return e;
        if (timed) timer_begin(*timed, "lap_moments", (double)N * (8 + 1 + 4 + sizeof(T)), st, &slot);
        if (tperm)   // t in band order (plans of fl_plan_laplace)
            k_lap_moments_sorted<T><<<nblocks, kLapWarps * 32, smem, st>>>(
                N, t, tband, tperm, c, P.levels, P.q, P.xi1, cheb, partial);
        else
            kern<<<nblocks, kLapWarps * 32, smem, st>>>(N, t, tband, c, P.levels, P.q, P.xi1, cheb,
                                                        partial);
        if (timed) timer_end(*timed, slot, st);
        k_lap_reduce<T><<<(entries * 32 + 255) / 256, 256, 0, st>>>(nblocks, entries, partial, vS);
    } else {
        cudaError_t e = cudaMemsetAsync(vS, 0, entries * sizeof(double), st);
        if (e != cudaSuccess) return e;
    }
    if (Kt)
        k_lap_couple_tab<<<std::max(1, P.levels - 1), 32 * std::min(P.q, 32), 0, st>>>(
            P.levels, P.q, ell, koff, Kt, vS, h, g);
    else
        k_lap_couple<<<std::max(1, P.levels - 1), std::max(32, ((P.q + 31) / 32) * 32), 0, st>>>(
            P.levels, P.q, P.y1, P.xi1, ell, cheb, vS, h, g);
    if (M > 0) {
        if (timed) timer_begin(*timed, "lap_eval", (double)M * (8 + 1 + sizeof(T)), st, &slot);
        k_lap_eval<T, BANDS_FROM_VALUES><<<(unsigned)((M + 255) / 256), 256, 0, st>>>(
            M, s, sband, P.levels, P.q, P.y1, cheb, h, g, f);
        if (timed) timer_end(*timed, slot, st);
    }
    if (timed) timed->launches += (N > 0 ? 2 : 0) + 1 + (M > 0 ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace fl

using namespace fl;

static fl_status lap_fail(fl_status s, const std::string& m) { return set_error(s, m); }

namespace fl {

// Moment tables per block for the generalised algorithm: up to kLapWarps, as
// many as fit 200 KB of shared memory (0: the tables do not fit).
static int gen_moment_warps(int entries, size_t tsize) {
    const size_t per = (size_t)entries * tsize;
    return (int)std::min<size_t>(kLapWarps, (size_t)(200 * 1024) / per);
}

template <typename T>
static cudaError_t gen_run(Plan& p, const T* c, T* f, cudaStream_t st) {
    const LapLayout L = lap_layout(p.levels, p.q, p.lap_blocks, sizeof(T));
    const int entries = (p.levels + 1) * (p.q + 1);
    unsigned char* scratch = (unsigned char*)p.d_lap;
    T* partial = (T*)(scratch + L.partial);
    double* vS = (double*)(scratch + L.vS);
    double* h = (double*)(scratch + L.h);
    const int nw = gen_moment_warps(entries, sizeof(T));
    const size_t smem = (size_t)nw * entries * sizeof(T);
    int slot = -1;
    if (p.N > 0 && p.levels > 1) {
        cudaError_t e = cudaFuncSetAttribute(k_lap_moments_sorted<T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        timer_begin(p, "lap_moments", (double)p.N * (8 + 1 + 4 + sizeof(T)), st, &slot);
        k_lap_moments_sorted<T><<<p.lap_blocks, nw * 32, smem, st>>>(
            p.N, p.d_ts, p.d_tbs, p.d_tperm, c, p.levels, p.q, p.xi1, p.d_cheb, partial);
        timer_end(p, slot, st);
        k_lap_reduce<T><<<(entries * 32 + 255) / 256, 256, 0, st>>>(p.lap_blocks, entries, partial, vS);
        k_gen_couple<<<p.levels - 1, 32 * std::min(p.q, 32), 0, st>>>(p.levels, p.q, p.d_lapK, vS, h);
        p.launches += 3;
    }
    if (p.M > 0) {
        timer_begin(p, "lap_eval", (double)p.M * (8 + 1 + sizeof(T)), st, &slot);
        if (p.lap_kernel == 2)
            k_gen_eval<T, 2><<<(unsigned)((p.M + 255) / 256), 256, 0, st>>>(
                p.M, p.d_s, p.d_sband, p.levels, p.q, p.y1, p.d_cheb, h, p.N, p.d_t, c, p.d_nearT,
                p.n_nearT, f);
        else
            k_gen_eval<T, 1><<<(unsigned)((p.M + 255) / 256), 256, 0, st>>>(
                p.M, p.d_s, p.d_sband, p.levels, p.q, p.y1, p.d_cheb, h, p.N, p.d_t, c, p.d_nearT,
                p.n_nearT, f);
        timer_end(p, slot, st);
        p.launches += 1;
    }
    return cudaGetLastError();
}

cudaError_t run_laplace(Plan& p, const void* c, void* f, cudaStream_t st) {
    if (p.lap_kernel != 0)
        return p.prec == FL_FP64 ? gen_run<double>(p, (const double*)c, (double*)f, st)
                                 : gen_run<float>(p, (const float*)c, (float*)f, st);
    LapParams P;
    memset(&P, 0, sizeof(P));
    P.q = p.q;
    P.levels = p.levels;
    P.y1 = p.y1;
    P.xi1 = p.xi1;
    for (int m = 1; m < p.levels && m < (int)p.bands.size(); ++m) P.ell[m] = p.bands[m].ell;
    if (p.prec == FL_FP64)
        return lap_run<double>(p.N, p.M, p.d_ts, p.d_s, p.d_tbs, p.d_sband, P, p.d_cheb,
                               (const double*)c, (double*)f, (unsigned char*)p.d_lap, p.lap_blocks,
                               st, &p, p.d_lapK, p.d_lapKoff, p.d_tperm);
    return lap_run<float>(p.N, p.M, p.d_ts, p.d_s, p.d_tbs, p.d_sband, P, p.d_cheb, (const float*)c,
                          (float*)f, (unsigned char*)p.d_lap, p.lap_blocks, st, &p, p.d_lapK,
                          p.d_lapKoff, p.d_tperm);
}

}  // namespace fl

#define LAP_CUDA(call, where)                                                      \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return lap_fail(e_ == cudaErrorMemoryAllocation ? FL_ENOMEM : FL_ECUDA, \
                            std::string(where) + ": " + cudaGetErrorString(e_));   \
    } while (0)

__global__ void k_lap_sortprep(int64_t n, const uint8_t* __restrict__ band, uint32_t* __restrict__ keys,
                               int32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        keys[i] = band[i];
        vals[i] = (int32_t)i;
    }
}

__global__ void k_lap_sorted(int64_t n, const double* __restrict__ t, const uint32_t* __restrict__ keys,
                             const int32_t* __restrict__ vals, double* __restrict__ ts,
                             uint8_t* __restrict__ bs, int32_t* __restrict__ perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        ts[i] = t[vals[i]];
        bs[i] = (uint8_t)keys[i];
        perm[i] = vals[i];
    }
}

// Plan time: copies of the t_k and their bands in band order (stable: equal
// bands keep the input order), with tperm the original index of each.
static cudaError_t sort_t_by_band(Plan& p, cudaStream_t st) {
    const int64_t n = p.N;
    uint32_t *keys = nullptr, *ktmp = nullptr, *hist = nullptr;
    int32_t *vals = nullptr, *vtmp = nullptr;
    double* ts = nullptr;
    uint8_t* bs = nullptr;
    const int64_t nblocks = (n + 2047) / 2048;        // radix-sort tiles of 256 x 8
    cudaError_t e = cudaMalloc((void**)&keys, n * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ktmp, n * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&vals, n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&vtmp, n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&hist, 256 * nblocks * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p.d_ts, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p.d_tbs, n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p.d_tperm, n * sizeof(int32_t));
    ts = p.d_ts;
    bs = p.d_tbs;
    if (e == cudaSuccess) {
        k_lap_sortprep<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, p.d_tband, keys, vals);
        e = radix_sort_pairs(keys, vals, ktmp, vtmp, hist, n, 8, st);
    }
    if (e == cudaSuccess) {
        k_lap_sorted<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, p.d_t, keys, vals, ts, bs, p.d_tperm);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (void* ptr : {(void*)keys, (void*)ktmp, (void*)vals, (void*)vtmp, (void*)hist}) cudaFree(ptr);
    return e;   // on failure the plan's destructor frees what was allocated
}

static fl_status plan_laplace_impl(Plan& p, const double* t, const double* s, int q,
                                   cudaStream_t st) {
    // interval ends and validity
    unsigned long long* dmx = nullptr;
    int* dflag = nullptr;
    LAP_CUDA(cudaMalloc((void**)&dmx, 2 * sizeof(unsigned long long)), "cudaMalloc");
    cudaError_t e = cudaMalloc((void**)&dflag, sizeof(int));
    unsigned long long mx[2] = {0, 0};
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(dmx, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dflag, 0, sizeof(int), st);
    if (e == cudaSuccess && (p.N > 0 || p.M > 0)) {
        k_lap_minmax<<<256, 256, 0, st>>>(p.N, t, p.M, s, dmx, dflag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(mx, dmx, sizeof(mx), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dmx);
    cudaFree(dflag);
    LAP_CUDA(e, "fl_plan_laplace: node scan");
    if (flag) return lap_fail(FL_EINVAL, "fl_plan_laplace: a t_k or s_j is negative or not finite");
    double xi1, y1;
    memcpy(&xi1, &mx[0], sizeof(double));
    memcpy(&y1, &mx[1], sizeof(double));
    LapParams P;
    if (!lap_params(p.eps, q, y1, xi1, &P))
        return lap_fail(FL_EUNSUPPORTED, "fl_plan_laplace: more than 127 levels or q above 40");
    p.q = P.q;
    p.levels = P.levels;
    p.y1 = y1;
    p.xi1 = xi1;
    p.eps_K = p.eps;
    p.bands.assign(P.levels + 1, BandHost());
    for (int m = 1; m < P.levels; ++m) {
        p.bands[m].ell = P.ell[m];
        p.bands[m].Lm = P.levels - m;
    }
    // copies of the nodes and their band ids
    const size_t N = (size_t)p.N, M = (size_t)p.M;
    if (N) {
        LAP_CUDA(cudaMalloc((void**)&p.d_t, N * sizeof(double)), "cudaMalloc t");
        LAP_CUDA(cudaMemcpyAsync(p.d_t, t, N * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy t");
        LAP_CUDA(cudaMalloc((void**)&p.d_tband, N), "cudaMalloc t bands");
        k_lap_band<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(p.N, p.d_t, xi1, P.levels, p.d_tband);
        LAP_CUDA(sort_t_by_band(p, st), "fl_plan_laplace: band order");
    }
    if (M) {
        LAP_CUDA(cudaMalloc((void**)&p.d_s, M * sizeof(double)), "cudaMalloc s");
        LAP_CUDA(cudaMemcpyAsync(p.d_s, s, M * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy s");
        LAP_CUDA(cudaMalloc((void**)&p.d_sband, M), "cudaMalloc s bands");
        k_lap_band<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(p.M, p.d_s, y1, P.levels, p.d_sband);
    }
    LAP_CUDA(cudaMalloc((void**)&p.d_cheb, 2 * kMaxQ * sizeof(double)), "cudaMalloc cheb");
    k_lap_cheb<<<1, 64, 0, st>>>(P.q, p.d_cheb);
    p.lap_blocks = lap_blocks(p.N);
    const size_t tsz = p.prec == FL_FP64 ? 8 : 4;
    if ((size_t)kLapWarps * (P.levels + 1) * (P.q + 1) * tsz > 200 * 1024)
        return lap_fail(FL_EUNSUPPORTED, "fl_plan_laplace: moment tables exceed shared memory "
                                         "(too many levels for this q)");
    const LapLayout L = lap_layout(P.levels, P.q, p.lap_blocks, p.prec == FL_FP64 ? 8 : 4);
    LAP_CUDA(cudaMalloc(&p.d_lap, L.total), "cudaMalloc scratch");
    std::vector<int> ell(P.levels + 1, 0);
    for (int m = 1; m < P.levels; ++m) ell[m] = P.ell[m];
    LAP_CUDA(cudaMemcpyAsync((unsigned char*)p.d_lap + L.ell, ell.data(), ell.size() * sizeof(int),
                             cudaMemcpyHostToDevice, st),
             "copy l_m");
    // coupling blocks K^{Y_m, Omega_l}, l = l_m .. L_m, as a table
    std::vector<int64_t> koff(P.levels + 1, 0);
    int64_t ktot = 0;
    for (int m = 1; m < P.levels; ++m) {
        koff[m] = ktot;
        ktot += (int64_t)std::max(0, P.levels - m - P.ell[m] + 1) * P.q * P.q;
    }
    if (ktot > 0) {
        LAP_CUDA(cudaMalloc((void**)&p.d_lapK, ktot * sizeof(double)), "cudaMalloc coupling table");
        LAP_CUDA(cudaMalloc((void**)&p.d_lapKoff, koff.size() * sizeof(int64_t)), "cudaMalloc coupling offsets");
        LAP_CUDA(cudaMemcpyAsync(p.d_lapKoff, koff.data(), koff.size() * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, st),
                 "copy coupling offsets");
        k_lap_ktable<<<P.levels - 1, 256, 0, st>>>(P.levels, P.q, y1, xi1,
                                                   (const int*)((unsigned char*)p.d_lap + L.ell),
                                                   p.d_lapKoff, p.d_cheb, p.d_lapK);
    }
    LAP_CUDA(cudaGetLastError(), "fl_plan_laplace: launch");
    LAP_CUDA(cudaStreamSynchronize(st), "fl_plan_laplace: synchronise");
    const size_t ts = p.prec == FL_FP64 ? 8 : 4;
    p.scratch_bytes = (double)L.total + N * 9.0 + M * 9.0;
    p.model_bytes = (double)N * (8 + 1 + ts) + (double)M * (8 + 1 + ts);
    return FL_OK;
}

// Generalised Algorithm 1: rank from the block bound of the proof of
// Theorem 3.1, C mu^q q^nu 2^(1-2q) (2 + (2/pi) ln q) (dist(A,0) dist(B,0))^-s
// <= eps, with dist(A,0) dist(B,0) >= (y_1 / 2^(M-1)) (xi_1 / 2^(M-1)) and the
// asymptotic-smoothness constants of the kernel (exp: C = 1, mu = 1, nu = 0,
// s = 0; K_1/2: C = sqrt(pi/2), mu = 1, nu = 0, s = 1/2).
static int gen_rank(int kind, double eps, double dmin) {
    const double C = kind == 2 ? sqrt(M_PI / 2.0) : 1.0, sexp = kind == 2 ? 0.5 : 0.0;
    for (int q = 1; q <= kGenMaxQ; ++q) {
        const double b = C * pow(2.0, 1 - 2 * q) * (2.0 + 2.0 / M_PI * log((double)q)) * pow(dmin, -sexp);
        if (b <= eps) return q;
    }
    return kGenMaxQ + 1;
}

static fl_status plan_general_impl(Plan& p, int kind, const double* t, const double* s, int q,
                                   cudaStream_t st) {
    unsigned long long* dmx = nullptr;
    int* dflag = nullptr;
    LAP_CUDA(cudaMalloc((void**)&dmx, 2 * sizeof(unsigned long long)), "cudaMalloc");
    cudaError_t e = cudaMalloc((void**)&dflag, 2 * sizeof(int));
    unsigned long long mx[2] = {0, 0};
    int flag[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemsetAsync(dmx, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dflag, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess && (p.N > 0 || p.M > 0)) {
        k_lap_minmax<<<256, 256, 0, st>>>(p.N, t, p.M, s, dmx, dflag);
        if (kind == 2) k_gen_positive<<<256, 256, 0, st>>>(p.N, t, p.M, s, dflag + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(mx, dmx, sizeof(mx), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flag, dflag, sizeof(flag), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dmx);
    cudaFree(dflag);
    LAP_CUDA(e, "fl_plan_kernel: node scan");
    if (flag[0]) return lap_fail(FL_EINVAL, "fl_plan_kernel: a t_k or s_j is negative or not finite");
    if (flag[1]) return lap_fail(FL_EINVAL, "fl_plan_kernel: the K_1/2 kernel needs every t_k, s_j > 0");
    double xi1, y1;
    memcpy(&xi1, &mx[0], sizeof(double));
    memcpy(&y1, &mx[1], sizeof(double));
    int levels = 1;
    if (y1 > 0.0 && xi1 > 0.0 && p.N > 0)
        levels = (int)std::max(1.0, ceil(log2(y1 * xi1 * (double)p.N / p.eps)) + 1.0);
    if (levels > 127) return lap_fail(FL_EUNSUPPORTED, "fl_plan_kernel: more than 127 levels");
    const double dmin = ldexp(y1, 1 - levels) * ldexp(xi1, 1 - levels);
    const int qq = q > 0 ? q : gen_rank(kind, p.eps, dmin);
    if (qq > kGenMaxQ) return lap_fail(FL_EUNSUPPORTED, "fl_plan_kernel: rank above 64 for this eps");
    p.lap_kernel = kind;
    p.q = qq;
    p.levels = levels;
    p.y1 = y1;
    p.xi1 = xi1;
    p.eps_K = p.eps;
    p.bands.assign(levels + 1, BandHost());
    const size_t N = (size_t)p.N, M = (size_t)p.M;
    if (N) {
        LAP_CUDA(cudaMalloc((void**)&p.d_t, N * sizeof(double)), "cudaMalloc t");
        LAP_CUDA(cudaMemcpyAsync(p.d_t, t, N * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy t");
        LAP_CUDA(cudaMalloc((void**)&p.d_tband, N), "cudaMalloc t bands");
        k_lap_band<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(p.N, p.d_t, xi1, levels, p.d_tband);
        LAP_CUDA(sort_t_by_band(p, st), "fl_plan_kernel: band order");
    }
    if (M) {
        LAP_CUDA(cudaMalloc((void**)&p.d_s, M * sizeof(double)), "cudaMalloc s");
        LAP_CUDA(cudaMemcpyAsync(p.d_s, s, M * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy s");
        LAP_CUDA(cudaMalloc((void**)&p.d_sband, M), "cudaMalloc s bands");
        k_lap_band<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(p.M, p.d_s, y1, levels, p.d_sband);
    }
    LAP_CUDA(cudaMalloc((void**)&p.d_cheb, 2 * kGenMaxQ * sizeof(double)), "cudaMalloc cheb");
    k_lap_cheb<<<1, kGenMaxQ, 0, st>>>(qq, p.d_cheb);
    p.lap_blocks = lap_blocks(p.N);
    const size_t tsz = p.prec == FL_FP64 ? 8 : 4;
    if (gen_moment_warps((levels + 1) * (qq + 1), tsz) < 1)
        return lap_fail(FL_EUNSUPPORTED, "fl_plan_kernel: moment tables exceed shared memory");
    const LapLayout L = lap_layout(levels, qq, p.lap_blocks, tsz);
    LAP_CUDA(cudaMalloc(&p.d_lap, L.total), "cudaMalloc scratch");
    // the Omega_M near field: indices of the t_k in the last frequency band
    if (N && levels > 1) {
        std::vector<uint8_t> tb(N);
        LAP_CUDA(cudaMemcpyAsync(tb.data(), p.d_tband, N, cudaMemcpyDeviceToHost, st), "copy t bands");
        LAP_CUDA(cudaStreamSynchronize(st), "fl_plan_kernel: synchronise");
        std::vector<int32_t> near;
        for (size_t k = 0; k < N; ++k)
            if (tb[k] == levels) near.push_back((int32_t)k);
        p.n_nearT = (int64_t)near.size();
        if (!near.empty()) {
            LAP_CUDA(cudaMalloc((void**)&p.d_nearT, near.size() * sizeof(int32_t)), "cudaMalloc near field");
            LAP_CUDA(cudaMemcpyAsync(p.d_nearT, near.data(), near.size() * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, st),
                     "copy near field");
        }
        const int64_t ktot = (int64_t)(levels - 1) * (levels - 1) * qq * qq;
        LAP_CUDA(cudaMalloc((void**)&p.d_lapK, ktot * sizeof(double)), "cudaMalloc coupling table");
        k_gen_ktable<<<levels - 1, 256, 0, st>>>(kind, levels, qq, y1, xi1, p.d_cheb, p.d_lapK);
    }
    LAP_CUDA(cudaGetLastError(), "fl_plan_kernel: launch");
    LAP_CUDA(cudaStreamSynchronize(st), "fl_plan_kernel: synchronise");
    p.scratch_bytes = (double)L.total + N * 9.0 + M * 9.0 +
                      (levels > 1 ? (double)(levels - 1) * (levels - 1) * qq * qq * 8.0 : 0.0);
    p.model_bytes = (double)N * (8 + 1 + tsz) + (double)M * (8 + 1 + tsz);
    return FL_OK;
}

extern "C" {

fl_status fl_plan_laplace(fl_plan_t* out, int64_t N, int64_t M, const double* t_dev,
                          const double* s_dev, int q, double eps, fl_precision prec, void* stream) {
    clear_error();
    if (!out) return lap_fail(FL_EINVAL, "fl_plan_laplace: out is NULL");
    *out = nullptr;
    if (N < 0 || M < 0) return lap_fail(FL_EINVAL, "fl_plan_laplace: need N >= 0 and M >= 0");
    if (N > ((int64_t)1 << 31) - 1 || M > ((int64_t)1 << 31) - 1)
        return lap_fail(FL_EUNSUPPORTED, "fl_plan_laplace: N or M above 2^31 - 1");
    if (!(eps > 0.0 && eps < 1.0)) return lap_fail(FL_EINVAL, "fl_plan_laplace: eps must lie in (0, 1)");
    if (q < 0 || q > kMaxQ) return lap_fail(FL_EINVAL, "fl_plan_laplace: q must lie in [0, 40]");
    if (prec != FL_FP32 && prec != FL_FP64) return lap_fail(FL_EINVAL, "fl_plan_laplace: unknown precision");
    if ((N > 0 && !t_dev) || (M > 0 && !s_dev)) return lap_fail(FL_EINVAL, "fl_plan_laplace: NULL nodes");
    fl_plan_s* h = new (std::nothrow) fl_plan_s();
    if (!h) return lap_fail(FL_ENOMEM, "fl_plan_laplace: host allocation");
    h->p.kind = 1;
    h->p.prec = prec;
    h->p.N = N;
    h->p.M = M;
    h->p.eps = eps;
    fl_status s = plan_laplace_impl(h->p, t_dev, s_dev, q, (cudaStream_t)stream);
    if (s != FL_OK) {
        delete h;
        return s;
    }
    *out = h;
    return FL_OK;
}

fl_status fl_plan_kernel(fl_plan_t* out, int kernel, int64_t N, int64_t M, const double* t_dev,
                         const double* s_dev, int q, double eps, fl_precision prec, void* stream) {
    clear_error();
    if (kernel == FL_KERNEL_LAPLACE) return fl_plan_laplace(out, N, M, t_dev, s_dev, q, eps, prec, stream);
    if (!out) return lap_fail(FL_EINVAL, "fl_plan_kernel: out is NULL");
    *out = nullptr;
    if (kernel != FL_KERNEL_EXP_GENERAL && kernel != FL_KERNEL_BESSEL_K_HALF)
        return lap_fail(FL_EINVAL, "fl_plan_kernel: unknown kernel");
    if (N < 0 || M < 0) return lap_fail(FL_EINVAL, "fl_plan_kernel: need N >= 0 and M >= 0");
    if (N > ((int64_t)1 << 31) - 1 || M > ((int64_t)1 << 31) - 1)
        return lap_fail(FL_EUNSUPPORTED, "fl_plan_kernel: N or M above 2^31 - 1");
    if (!(eps > 0.0 && eps < 1.0)) return lap_fail(FL_EINVAL, "fl_plan_kernel: eps must lie in (0, 1)");
    if (q < 0 || q > kGenMaxQ) return lap_fail(FL_EINVAL, "fl_plan_kernel: q must lie in [0, 64]");
    if (prec != FL_FP32 && prec != FL_FP64) return lap_fail(FL_EINVAL, "fl_plan_kernel: unknown precision");
    if ((N > 0 && !t_dev) || (M > 0 && !s_dev)) return lap_fail(FL_EINVAL, "fl_plan_kernel: NULL nodes");
    fl_plan_s* h = new (std::nothrow) fl_plan_s();
    if (!h) return lap_fail(FL_ENOMEM, "fl_plan_kernel: host allocation");
    h->p.kind = 1;
    h->p.prec = prec;
    h->p.N = N;
    h->p.M = M;
    h->p.eps = eps;
    fl_status s = plan_general_impl(h->p, kernel, t_dev, s_dev, q, (cudaStream_t)stream);
    if (s != FL_OK) {
        delete h;
        return s;
    }
    *out = h;
    return FL_OK;
}

fl_status fl_laplace_real(fl_plan_t h, const void* c_dev, void* f_dev, void* stream) {
    clear_error();
    if (!h || h->p.kind != 1) return lap_fail(FL_EINVAL, "fl_laplace_real: not a Laplace plan");
    if ((h->p.N > 0 && !c_dev) || (h->p.M > 0 && !f_dev))
        return lap_fail(FL_EINVAL, "fl_laplace_real: NULL buffer");
    cudaError_t e = run_laplace(h->p, c_dev, f_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return lap_fail(FL_ECUDA, std::string("fl_laplace_real: ") + cudaGetErrorString(e));
    return FL_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of fl_laplace_real (fl_laplace_real_noalloc).
//
// Some callers cannot allocate device memory at the point where they need the
// transform: code running inside another framework's memory pool that forbids
// outside allocations, real-time loops where a cudaMalloc (which may
// synchronise the device) is not allowed, or a device that is already full.
// For them every buffer this entry point uses beyond the caller's inputs and
// outputs lives in g_noalloc_scratch, one static device array of
// kNoAllocScratchBytes that each GPU loading libfl.so holds until the process
// exits.  Host code cannot pass the array's name to a kernel (on the host it
// is only a stand-in for the device symbol), so the first call on each device
// looks up its device address with cudaGetSymbolAddress, with that device
// current, and keeps it.
constexpr size_t kNoAllocScratchBytes = (size_t)2 << 20;   // 2 MiB per GPU

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kNoAllocMaxDevices = 64;

std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set up once).
fl_status noalloc_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return set_error(FL_ECUDA, std::string("fl_laplace_real_noalloc: cudaGetDevice: ") +
                                       cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return set_error(FL_EUNSUPPORTED, "fl_laplace_real_noalloc: device index above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(FL_ECUDA, std::string("fl_laplace_real_noalloc: cudaGetSymbolAddress: ") +
                                           cudaGetErrorString(e));
        g_noalloc_ptr[dev] = (unsigned char*)p;
    }
    *out = g_noalloc_ptr[dev];
    return FL_OK;
}

struct EllArg {
    int v[FL_MAX_LEVELS];
};

__global__ void k_store_ell(EllArg a, int n, int* __restrict__ dst) {
    const int i = threadIdx.x;
    if (i < n) dst[i] = a.v[i];
}

}  // namespace

extern "C" {

fl_status fl_laplace_real_noalloc(int64_t N, int64_t M, const double* t_dev, const double* s_dev,
                                  const void* c_dev, void* f_dev, int q, double eps,
                                  fl_precision prec, void* stream) {
    clear_error();
    if (N < 0 || M < 0) return lap_fail(FL_EINVAL, "fl_laplace_real_noalloc: need N >= 0 and M >= 0");
    if (N > ((int64_t)1 << 31) - 1 || M > ((int64_t)1 << 31) - 1)
        return lap_fail(FL_EUNSUPPORTED, "fl_laplace_real_noalloc: N or M above 2^31 - 1");
    if (!(eps > 0.0 && eps < 1.0))
        return lap_fail(FL_EINVAL, "fl_laplace_real_noalloc: eps must lie in (0, 1)");
    if (q < 0 || q > kMaxQ) return lap_fail(FL_EINVAL, "fl_laplace_real_noalloc: q must lie in [0, 40]");
    if (prec != FL_FP32 && prec != FL_FP64)
        return lap_fail(FL_EINVAL, "fl_laplace_real_noalloc: unknown precision");
    if ((N > 0 && (!t_dev || !c_dev)) || (M > 0 && (!s_dev || !f_dev)))
        return lap_fail(FL_EINVAL, "fl_laplace_real_noalloc: NULL buffer");
    unsigned char* scratch = nullptr;
    fl_status st0 = noalloc_scratch(&scratch);
    if (st0 != FL_OK) return st0;
    cudaStream_t st = (cudaStream_t)stream;

    // [0, 256): interval maxima (2 x u64) and the validity flag; cleared every call
    unsigned long long* dmx = (unsigned long long*)scratch;
    int* dflag = (int*)(scratch + 2 * sizeof(unsigned long long));
    LAP_CUDA(cudaMemsetAsync(scratch, 0, 256, st), "fl_laplace_real_noalloc: clear");
    if (N > 0 || M > 0) k_lap_minmax<<<256, 256, 0, st>>>(N, t_dev, M, s_dev, dmx, dflag);
    LAP_CUDA(cudaGetLastError(), "fl_laplace_real_noalloc: launch");
    unsigned long long mx[2] = {0, 0};
    int flag = 0;
    LAP_CUDA(cudaMemcpyAsync(mx, dmx, sizeof(mx), cudaMemcpyDeviceToHost, st), "fl_laplace_real_noalloc: read");
    LAP_CUDA(cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, st),
             "fl_laplace_real_noalloc: read");
    LAP_CUDA(cudaStreamSynchronize(st), "fl_laplace_real_noalloc: synchronise");
    if (flag) return lap_fail(FL_EINVAL, "fl_laplace_real_noalloc: a t_k or s_j is negative or not finite");
    double xi1, y1;
    memcpy(&xi1, &mx[0], sizeof(double));
    memcpy(&y1, &mx[1], sizeof(double));
    LapParams P;
    if (!lap_params(eps, q, y1, xi1, &P))
        return lap_fail(FL_EUNSUPPORTED, "fl_laplace_real_noalloc: more than 127 levels or q above 40");
    const size_t tsz = prec == FL_FP64 ? 8 : 4;
    if ((size_t)kLapWarps * (P.levels + 1) * (P.q + 1) * tsz > 200 * 1024)
        return lap_fail(FL_EUNSUPPORTED, "fl_laplace_real_noalloc: moment tables exceed shared memory");

    // [256, 256 + cheb): Chebyshev table; then the Algorithm 1 layout with the
    // partial sums of kLapMaxBlocks moment blocks reserved whatever N is, so
    // whether a problem fits depends on the number of levels and q alone
    const size_t cheb_off = 256;
    const size_t lap_off = align256(cheb_off + 2 * kMaxQ * sizeof(double));
    const int nblocks = lap_blocks(N);
    const LapLayout L = lap_layout(P.levels, P.q, kLapMaxBlocks, tsz);
    if (lap_off + L.total > kNoAllocScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "fl_laplace_real_noalloc: this problem needs %zu bytes of scratch (levels = %d, "
                 "q = %d); the static maximum is %zu bytes -- use fl_plan_laplace, a larger eps "
                 "or a smaller max(s) * max(t)",
                 lap_off + L.total, P.levels, P.q, kNoAllocScratchBytes);
        return lap_fail(FL_EUNSUPPORTED, msg);
    }
    double* cheb = (double*)(scratch + cheb_off);
    unsigned char* lap = scratch + lap_off;
    k_lap_cheb<<<1, 64, 0, st>>>(P.q, cheb);
    EllArg ea;
    for (int m = 0; m < FL_MAX_LEVELS; ++m) ea.v[m] = (m < P.levels) ? P.ell[m] : 0;
    k_store_ell<<<1, FL_MAX_LEVELS, 0, st>>>(ea, P.levels + 1, (int*)(lap + L.ell));
    LAP_CUDA(cudaGetLastError(), "fl_laplace_real_noalloc: launch");
    cudaError_t e;
    if (prec == FL_FP64)
        e = lap_run<double, true>(N, M, t_dev, s_dev, nullptr, nullptr, P, cheb, (const double*)c_dev,
                                  (double*)f_dev, lap, nblocks, st, nullptr, nullptr, nullptr, nullptr,
                                  kLapMaxBlocks);
    else
        e = lap_run<float, true>(N, M, t_dev, s_dev, nullptr, nullptr, P, cheb, (const float*)c_dev,
                                 (float*)f_dev, lap, nblocks, st, nullptr, nullptr, nullptr, nullptr,
                                 kLapMaxBlocks);
    LAP_CUDA(e, "fl_laplace_real_noalloc");
    return FL_OK;
}

}  // extern "C"
