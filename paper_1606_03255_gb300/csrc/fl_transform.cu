// fl_transform.cu -- the kernels of Algorithm 2 (Kunis & Melzer, Section 4) and
// of its adjoint.
//
// For a band Y_m of nodes the paper evaluates (Algorithm 2, Lemma 4.2)
//
//   f~_j = sum_s L_s^{Y_m}(y_j) * [A~ (c (.) W_{.,s})](x_j),
//   W_{k,s} = sum_r K^{Y_m,Omega_l}_{s r} L_r^{Omega_l}(k)   for l_m <= l(k) <= L_m,
//   W_{k,s} = 1  for l(k) > L_m (region (iv); folded into every s since
//               sum_s L_s = 1),   W_{k,s} = 0 for l(k) < l_m (region (ii)),
//
// where A~ is one NFFT with q right-hand sides.  Each NFFT here is:
//   deconvolution  g^_k' = c_k W_{k,s} / Phi(k'/n)      (folded into table D)
//   FFT            g_l = sum_k' g^_k' exp(+2 pi i k' l / n)
//   window gather  s(x) = sum_l g_l phi(n x - l),  Kaiser-Bessel phi, 2 m_w taps
// with centred frequencies k' = k - N_m/2 and the shift exp(pi i N_m x) applied
// after the gather.  The band's q results are recombined with the barycentric
// weights L_s^{Y_m}(y_j) (Section 2) in the same gather kernel.
#include <math.h>

#include "fl_fft.cuh"
#include "fl_ffmath.cuh"

namespace fl {
FL_FFT_EXTERN(float)
FL_FFT_EXTERN(double)
FL_FFT_EXTERN_FF
}  // namespace fl

namespace fl {

constexpr double kPi = 3.141592653589793238462643383279;
constexpr double kTwoPiD = 6.283185307179586476925286766559;

// ---------------------------------------------------------------------------
// Tables (plan time).

__device__ __forceinline__ int band_of_freq(double k, double xi1, int levels) {
    if (levels <= 1) return 1;
    if (k > ldexp(xi1, -1)) return 1;
    if (!(k > ldexp(xi1, -(levels - 1)))) return levels;
    int b = (int)floor(log2(xi1 / k)) + 1;
    b = max(1, min(b, levels - 1));
    while (b > 1 && k > ldexp(xi1, -(b - 1))) --b;
    while (b < levels - 1 && !(k > ldexp(xi1, -b))) ++b;
    return b;
}

// Chebyshev points t_s = cos((2s+1) pi / (2q)) and barycentric weights
// lambda_s = (-1)^s sin((2s+1) pi / (2q)) (Section 2); cheb32 holds t_s as a
// float pair (hi, lo: t_s = hi + lo to ~2^-48), lambda_s in float, and the
// low part of lambda_s (lambda_s = cheb32[2q + s] + cheb32[3q + s] to ~2^-48).
__global__ void k_cheb(int q, double* cheb, float* cheb32) {
    const int s = threadIdx.x;
    if (s >= q) return;
    double sn, cs;
    sincospi((2.0 * s + 1.0) / (2.0 * q), &sn, &cs);
    cheb[s] = cs;
    cheb[q + s] = (s & 1) ? -sn : sn;
    const float hi = (float)cs;
    cheb32[s] = hi;
    cheb32[q + s] = (float)(cs - (double)hi);
    cheb32[2 * q + s] = (float)cheb[q + s];
    cheb32[3 * q + s] = (float)(cheb[q + s] - (double)cheb32[2 * q + s]);
}

// K^{Y_m,Omega_l}_{s r} = exp(-y_s^{Y_m} xi_r^{Omega_l}) for l = l_m..L_m
// (Definition 3.2), written as Kt[(l - l_m) q^2 + s q + r].
__global__ void k_coupling(double y1, double xi1, int m, int ellm, int Lm, int q,
                           const double* __restrict__ cheb, double* __restrict__ Kt) {
    const int nl = Lm - ellm + 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nl * q * q) return;
    const int r = (int)(i % q), s = (int)((i / q) % q), l = ellm + (int)(i / ((int64_t)q * q));
    const double ay = ldexp(y1, -m), ax = ldexp(xi1, -l);
    const double ys = 1.5 * ay + 0.5 * ay * cheb[s];
    const double xr = 1.5 * ax + 0.5 * ax * cheb[r];
    Kt[i] = exp(-ys * xr);
}

// D[s K + k] = W_{k,s} / Phi(k'/n), k' = k - N_m/2, with the Kaiser-Bessel
// transform Phi(nu) = pi I_0(m_w sqrt(b^2 - (2 pi nu)^2)) (window in grid units).
// one_sided: W_{k,s} = exp(-y_s k) at the band's Chebyshev points y_s (the
// interpolation in y alone, first term of the proof of Theorem 3.1).
// xis (real exponents): frequency k is the sorted exponent xis[k], no 1/Phi
// is folded in (the NNFFT deconvolves per grid frequency instead), and the
// table is exponent-major, D[k dld + s] (B.dld > 0).
template <typename T>
__global__ void k_weights(BandDev B, int ellm, int Lm, int q, double xi1, int levels,
                          const double* __restrict__ cheb, const double* __restrict__ Kt,
                          int mw, double kb_b, int one_sided, const double* __restrict__ xis,
                          T* __restrict__ D) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B.K) return;
    const double xk = xis ? xis[k] : (double)(B.k0 + k);   // the band's (sub-band's) frequency
    double inv_phi = 1.0;
    if (!xis) {   // the window of this grid: shape B.kb (kb_b for sigma = 2)
        const double nu = (double)(k - B.Nm / 2) / (double)B.n;
        const double arg = B.kb * B.kb - (kTwoPiD * nu) * (kTwoPiD * nu);
        inv_phi = 1.0 / (kPi * cyl_bessel_i0((double)mw * sqrt(fmax(arg, 0.0))));
    }
    // entry s of frequency k at Dk[s * ds]
    T* Dk = D + B.D_off + (B.dld ? k * B.dld : k);
    const int64_t ds = B.dld ? 1 : B.K;
    if (B.nrhs == 1) {
        Dk[0] = (T)inv_phi;
        return;
    }
    if (one_sided) {
        for (int s = 0; s < q; ++s) {
            const double ys = B.yc + B.yh * cheb[s];
            Dk[s * ds] = (T)(exp(-ys * xk) * inv_phi);
        }
        return;
    }
    const int l = band_of_freq(xk, xi1, levels);
    if (l > Lm) {   // region (iv): kernel ~ 1
        for (int s = 0; s < q; ++s) Dk[s * ds] = (T)inv_phi;
        return;
    }
    if (l < ellm) {   // region (ii): kernel ~ 0 (not reached: k < K)
        for (int s = 0; s < q; ++s) Dk[s * ds] = (T)0;
        return;
    }
    // Lagrange weights L_r^{Omega_l}(k), barycentric form, tau in [-1, 1]
    const double ax = ldexp(xi1, -l);
    const double tau = (xk - 1.5 * ax) / (0.5 * ax);
    double Lr[kMaxQ];
    int hit = -1;
    double den = 0.0;
    for (int r = 0; r < q; ++r) {
        const double d = tau - cheb[r];
        if (d == 0.0) hit = r;
        Lr[r] = cheb[q + r] / d;
        den += Lr[r];
    }
    for (int r = 0; r < q; ++r) Lr[r] = (hit >= 0) ? (r == hit ? 1.0 : 0.0) : Lr[r] / den;
    const double* Kb = Kt + (int64_t)(l - ellm) * q * q;
    for (int s = 0; s < q; ++s) {
        double W = 0.0;
        for (int r = 0; r < q; ++r) W += Kb[s * q + r] * Lr[r];
        Dk[s * ds] = (T)(W * inv_phi);
    }
}

template <typename T>
static cudaError_t build_tables_t(Plan& p, const Instance& in, cudaStream_t st) {
    double* Kt = nullptr;
    cudaError_t e = cudaSuccess;
    int64_t kt_max = 0;
    for (int lb = 1; lb <= in.levels; ++lb) {
        const BandHost& bh = p.bands[in.band_base + lb];
        if (bh.dev.route != 1 || bh.dev.nrhs == 1 || p.variant == 1) continue;
        kt_max = std::max<int64_t>(kt_max, (int64_t)(bh.Lm - bh.ell + 1) * p.q * p.q);
    }
    if (kt_max > 0) {
        e = cudaMallocAsync((void**)&Kt, kt_max * sizeof(double), st);
        if (e != cudaSuccess) return e;
    }
    for (int lb = 1; lb <= in.levels; ++lb) {
        const BandHost& bh = p.bands[in.band_base + lb];
        if (bh.dev.route != 1) continue;
        if (bh.dev.nrhs > 1 && p.variant == 0) {
            const int64_t nk = (int64_t)(bh.Lm - bh.ell + 1) * p.q * p.q;
            k_coupling<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(p.y1, in.xi1, lb, bh.ell, bh.Lm,
                                                                     p.q, p.d_cheb, Kt);
        }
        // a split band: the weights of each sub-band's frequencies (same coupling blocks)
        for (int c = 0; c < std::max(1, bh.dev.nsub); ++c) {
            const BandDev& d = bh.dev.nsub > 0 ? p.bands[bh.dev.sub0 + c].dev : bh.dev;
            k_weights<T><<<(unsigned)((d.K + 255) / 256), 256, 0, st>>>(
                d, bh.ell, bh.Lm, p.q, in.xi1, in.levels, p.d_cheb, Kt, p.mw, p.kb_b, p.variant,
                p.xi_mode ? p.d_xis : nullptr, (T*)p.d_D);
        }
    }
    e = cudaGetLastError();
    if (Kt) {
        cudaError_t e2 = cudaFreeAsync(Kt, st);
        if (e == cudaSuccess) e = e2;
    }
    return e;
}

// Stage twiddles of the four-step passes (layout in fl_common.cuh): entry
// 2 NS p + 2 k + h of the stage of span NS = 2^d and radix R in region
// (LOG2L, FIRST) is exp(2 pi i r k / (NS R)) with r = 2p + 1 + h < R, computed in
// FP64 (exact argument: r k < NS R, a power of two) and rounded once to T.
// Unused entries are zero.
template <typename T>
__global__ void k_twiddles(C_t<T>* __restrict__ tw) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kTwEntries) return;
    const int region = (int)(i / kTwRegion), e = (int)(i % kTwRegion);
    const int LOG2L = kTwMinLog + region / 2, FIRST = 3 + region % 2;
    C_t<T> v{(T)0, (T)0};
    if (LOG2L > FIRST) {
        for (int d = FIRST; d < LOG2L; d += 4) {
            const int NS = 1 << d, R = 1 << tw_stage_log(LOG2L, FIRST, d);
            const int off = tw_off(LOG2L, FIRST, d);
            if (e >= off && e < off + R * NS) {
                const int rel = e - off, pr = rel / (2 * NS), rem = rel % (2 * NS);
                const int k = rem / 2, r = 2 * pr + 1 + rem % 2;
                if (r < R) {
                    double sn, cs;
                    sincospi(2.0 * (double)(r * k) / (double)(NS * R), &sn, &cs);
                    v = C_t<T>{(T)cs, (T)sn};
                }
            }
        }
    }
    tw[i] = v;
}

// Float pairs: the pass-1 output twiddles as products of two tables,
// tab[a] = exp(2 pi i a / 2^12) and tab[4096 + b] = exp(2 pi i b / 2^24),
// a, b < 4096, each computed in FP64 (exact arguments) and rounded once.
__global__ void k_ff_tables(ffc* __restrict__ tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8192) return;
    const double x = i < 4096 ? ldexp((double)i, -11) : ldexp((double)(i - 4096), -23);
    double sn, cs;
    sincospi(x, &sn, &cs);
    tab[i] = ffc{ff(cs), ff(sn)};
}

cudaError_t build_twiddles(Plan& p, cudaStream_t st) {
    const unsigned blocks = (unsigned)((kTwEntries + 255) / 256);
    if (p.prec == FL_FP64_FF) {
        k_twiddles<ff><<<blocks, 256, 0, st>>>((ffc*)p.d_tw);
        k_ff_tables<<<8192 / 256, 256, 0, st>>>((ffc*)p.d_tw + kTwEntries);
    } else if (p.prec == FL_FP64) {
        k_twiddles<double><<<blocks, 256, 0, st>>>((C_t<double>*)p.d_tw);
    } else {
        k_twiddles<float><<<blocks, 256, 0, st>>>((C_t<float>*)p.d_tw);
    }
    return cudaGetLastError();
}

// Per sorted node of an FP32 plan: X = x 2^64 with x = Re w mod 1 (exact for
// x >= 2^-11, within 2^-64 below), and tau = (2 pi Im w - y_c) / y_h of its
// band as a float pair (hi = tau rounded, lo = the rest), for gather_node_f32;
// for a node of a direct-route band y = 2 pi Im w as a float pair instead, for
// the direct kernels (no FP64 arithmetic per node there).
__global__ void k_node_tab(int64_t M, const double2* __restrict__ ws, const int32_t* __restrict__ bandid,
                           const BandDev* __restrict__ bands, uint4* __restrict__ tab) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const double2 wv = ws[i];
    const double x = wv.x - floor(wv.x);
    const uint64_t X = (uint64_t)ldexp(x, 64);
    const BandDev B = bands[bandid[i]];
    float th = 0.f, tl = 0.f;
    if (B.route == 2) {
        const double y = kTwoPiD * wv.y;
        th = (float)y;
        tl = (float)(y - (double)th);
    } else if (B.nrhs > 1) {
        const double tau = (kTwoPiD * wv.y - B.yc) * B.yh_inv;
        th = (float)tau;
        tl = (float)(tau - (double)th);
    }
    tab[i] = make_uint4((unsigned)X, (unsigned)(X >> 32), __float_as_uint(th), __float_as_uint(tl));
}

cudaError_t build_node_table(Plan& p, cudaStream_t st) {
    k_node_tab<<<(unsigned)((p.M + 255) / 256), 256, 0, st>>>(p.M, p.d_ws, p.d_bandid, p.d_bands, p.d_ntab);
    return cudaGetLastError();
}

cudaError_t build_cheb(Plan& p, cudaStream_t st) {
    k_cheb<<<1, 64, 0, st>>>(p.q, p.d_cheb, p.d_cheb32);
    return cudaGetLastError();
}

cudaError_t build_tables(Plan& p, const Instance& in, cudaStream_t st) {
    if (p.prec == FL_FP64_FF) return build_tables_t<ff>(p, in, st);
    return p.prec == FL_FP64 ? build_tables_t<double>(p, in, st) : build_tables_t<float>(p, in, st);
}

// ---------------------------------------------------------------------------
// Window and barycentric weights of one node.


// Barycentric weights of y in Y_m = [yc - yh, yc + yh]: tau - t_s in double (the
// cancellation-prone step), the rest in T.  Returns in Ls[0..q-1].
template <typename T>
__device__ __forceinline__ void bary_weights(double y, const BandDev& B, int q,
                                             const double* __restrict__ cheb, T* Ls) {
    const double tau = (y - B.yc) * B.yh_inv;
    T den = 0;
    int hit = -1;
    for (int s = 0; s < q; ++s) {
        const double d = tau - cheb[s];
        if (d == 0.0) hit = s;
        Ls[s] = (T)cheb[q + s] / (T)d;
        den += Ls[s];
    }
    const T inv = (T)1 / den;
    for (int s = 0; s < q; ++s) Ls[s] = (hit >= 0) ? (s == hit ? (T)1 : (T)0) : Ls[s] * inv;
}

// FP32 form of the q-right-hand-side gather: sum_s L_s(y) sum_t phi_t g_s[lo + t].
// The barycentric differences tau - t_s are formed from float pairs
// (tau_hi + tau_lo) - (t_s,hi + t_s,lo): the high parts cancel exactly when
// tau is near t_s (Sterbenz), so each difference keeps float relative accuracy
// without FP64 arithmetic per s.  The weights are recomputed in the gather loop
// instead of being stored, and two right-hand sides are gathered per step.
template <int MW>
__device__ __forceinline__ float2 gather_rhs_f32(const float2* __restrict__ g, const BandDev& B,
                                                 int64_t lo, int64_t nmask, const float* phi,
                                                 float th, float tl, int q,
                                                 const float* __restrict__ cheb32) {
    float den = 0.f;
    int hit = -1;
    for (int s = 0; s < q; ++s) {
        const float d = (th - cheb32[s]) + (tl - cheb32[q + s]);
        if (d == 0.f) hit = s;
        den += cheb32[2 * q + s] / d;
    }
    const float inv = 1.f / den;
    float2 acc = {0.f, 0.f};
    for (int s = 0; s < q; s += 2) {
        const bool two = s + 1 < q;
        const float2* g0 = g + (int64_t)s * B.n;
        const float2* g1 = g0 + B.n;
        float2 a0 = {0.f, 0.f}, a1 = {0.f, 0.f};
#pragma unroll
        for (int t = 0; t < 2 * MW; ++t) {
            const int64_t idx = (lo + t) & nmask;
            const float2 v0 = g0[idx];
            const float2 v1 = two ? g1[idx] : float2{0.f, 0.f};
            a0.x += phi[t] * v0.x;
            a0.y += phi[t] * v0.y;
            a1.x += phi[t] * v1.x;
            a1.y += phi[t] * v1.y;
        }
        const float d0 = (th - cheb32[s]) + (tl - cheb32[q + s]);
        float L0 = hit >= 0 ? (s == hit ? 1.f : 0.f) : cheb32[2 * q + s] / d0 * inv;
        float L1 = 0.f;
        if (two) {
            const float d1 = (th - cheb32[s + 1]) + (tl - cheb32[q + s + 1]);
            L1 = hit >= 0 ? (s + 1 == hit ? 1.f : 0.f) : cheb32[2 * q + s + 1] / d1 * inv;
        }
        acc.x += L0 * a0.x + L1 * a1.x;
        acc.y += L0 * a0.y + L1 * a1.y;
    }
    return acc;
}

// sum_t phi_t g[(lo + t) mod n] over the 2 m_w taps of one right-hand side.
template <int MW, typename T, typename C>
__device__ __forceinline__ C tap_sum(const C* __restrict__ g, int64_t lo, int64_t nmask, const T* phi) {
    C a = {(T)0, (T)0};
#pragma unroll
    for (int t = 0; t < 2 * MW; ++t) {
        const C v = g[(lo + t) & nmask];
        a.x += phi[t] * v.x;
        a.y += phi[t] * v.y;
    }
    return a;
}

// FP32 recombination of a node of a fused band (see k_pass2): its partial tap
// sums a_s = sum_p pp[s][jl P + p] over the row blocks its window spans, with
// the barycentric weights of gather_rhs_f32 (one right-hand side: a_0).
__device__ __forceinline__ float2 fused_rhs_f32(const float2* __restrict__ pp, const BandDev& B,
                                                int64_t jl, float th, float tl, int q,
                                                const float* __restrict__ cheb32) {
    const int P = B.pparts;
    const float2* a = pp + B.pp_off + jl * P;
    const int64_t stride = B.nodes * P;
    auto part_sum = [&](int s) {
        float2 v = {0.f, 0.f};
        for (int k = 0; k < P; ++k) {
            const float2 w = a[s * stride + k];
            v.x += w.x;
            v.y += w.y;
        }
        return v;
    };
    if (B.nrhs == 1) return part_sum(0);
    float den = 0.f;
    int hit = -1;
    for (int s = 0; s < q; ++s) {
        const float d = (th - cheb32[s]) + (tl - cheb32[q + s]);
        if (d == 0.f) hit = s;
        den += cheb32[2 * q + s] / d;
    }
    const float inv = 1.f / den;
    float2 acc = {0.f, 0.f};
    for (int s = 0; s < q; ++s) {
        const float d = (th - cheb32[s]) + (tl - cheb32[q + s]);
        const float L = hit >= 0 ? (s == hit ? 1.f : 0.f) : cheb32[2 * q + s] / d * inv;
        const float2 v = part_sum(s);
        acc.x += L * v.x;
        acc.y += L * v.y;
    }
    return acc;
}

// k x mod 1 in turns, in [-1/2, 1/2), for x held as the 64-bit fixed-point
// X = x 2^64 (exact) and an integer k: the wrapped product k X mod 2^64, whose
// top 24 bits as a signed value are the turns to 2^-24 (float resolution).
__device__ __forceinline__ float fixed_turns(uint64_t X, uint64_t k) {
    return (float)((int64_t)(k * X) >> 40) * 0x1p-24f;
}

// A split band (B.nsub > 0): the sum over its sub-bands S of
// exp(2 pi i kc_S x) times S's recombined partial sums, kc_S = S.k0 + S.Nm/2
// the sub-band's centre frequency.
__device__ __forceinline__ float2 split_rhs_f32(const float2* __restrict__ pp,
                                                const BandDev* __restrict__ bands, const BandDev& B,
                                                int64_t jl, float th, float tl, uint64_t X, int q,
                                                const float* __restrict__ cheb32) {
    float2 acc = {0.f, 0.f};
    for (int c = 0; c < B.nsub; ++c) {
        const BandDev S = bands[B.sub0 + c];
        const float2 a = fused_rhs_f32(pp, S, jl, th, tl, q, cheb32);
        const float ph = fixed_turns(X, (uint64_t)(S.k0 + (S.Nm >> 1)));
        acc = cadd(acc, cmul(a, expipi<float>(2.f * ph)));
    }
    return acc;
}

// The FP32 gather of one node from its plan-time record (x as X = x 2^64,
// the barycentric coordinate tau = (y - y_c) / y_h as a float pair): every
// phase reduction -- the grid cell and its fraction floor/frac(n x), the
// centring shift (N_m/2) x mod 1, a sub-band's kc x mod 1 -- is an exact
// shift or wrapped product of X, so no FP64 arithmetic runs per node.
template <int MW>
__device__ __forceinline__ float2 gather_node_f32(const uint4 nd, int64_t jl, const BandDev& B,
                                                  const BandDev* __restrict__ bands,
                                                  const float2* __restrict__ grid,
                                                  const float* __restrict__ cheb32, int q, float kb_b,
                                                  const float2* __restrict__ fpp) {
    const uint64_t X = ((uint64_t)nd.y << 32) | nd.x;
    const float th = __uint_as_float(nd.z), tl = __uint_as_float(nd.w);
    if (B.nsub > 0) return split_rhs_f32(fpp, bands, B, jl, th, tl, X, q, cheb32);
    float2 acc;
    if (B.fused) {
        acc = fused_rhs_f32(fpp, B, jl, th, tl, q, cheb32);
    } else {
        const int64_t u = (int64_t)(X >> (64 - B.log2n));
        const float fr = (float)((X << B.log2n) >> 40) * 0x1p-24f;
        const int64_t lo = u - (MW - 1);
        float phi[2 * MW];
#pragma unroll
        for (int t = 0; t < 2 * MW; ++t) phi[t] = kb_window<float>(fr + (float)(MW - 1 - t), (float)MW, kb_b);
        const float2* g = grid + B.grid_off;
        const int64_t nmask = B.n - 1;
        acc = B.nrhs > 1 ? gather_rhs_f32<MW>(g, B, lo, nmask, phi, th, tl, q, cheb32)
                         : tap_sum<MW>(g, lo, nmask, phi);
    }
    // centring shift exp(2 pi i (N_m/2) x), N_m a power of two
    return cmul(acc, expipi<float>(2.f * fixed_turns(X, (uint64_t)(B.Nm >> 1))));
}

// Gather + barycentric recombination + centring shift, one thread per node in
// sorted order; writes f[perm[i]].  Z^0 nodes (band 0) receive c_0.
// XI (real exponents): the outer NFFT of the band's NNFFT runs at x/2, Z^0
// nodes receive 0, and the epilogue is exp(2 pi i xc x) / Phi(x/2) instead of
// the centring shift.
template <typename T, int MW, bool XI = false>
__global__ void __launch_bounds__(256) k_gather(int64_t M, const double2* __restrict__ ws,
                                                const int32_t* __restrict__ perm,
                                                const int32_t* __restrict__ bandid,
                                                const BandDev* __restrict__ bands,
                                                const C_t<T>* __restrict__ grid,
                                                const double* __restrict__ cheb,
                                                const float* __restrict__ cheb32, int q, T kb_b,
                                                const C_t<T>* __restrict__ c, int deriv,
                                                const C_t<T>* __restrict__ rmul,
                                                const float2* __restrict__ fpp,
                                                const uint4* __restrict__ ntab,
                                                C_t<T>* __restrict__ f) {
    using C = C_t<T>;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int b = bandid[i];
    const int32_t j = perm[i];
    const BandDev B = bands[b];
    if (B.K == 0 && B.n == 0) {   // Z^0 (band 0 of its transform): c_0 (0 for real exponents >= 1)
        f[j] = (deriv || XI) ? C{(T)0, (T)0} : c[B.c_off];
        return;
    }
    // with rmul: f[j] = rmul[j] * conj(value) (node gradient, see fl_grad_w)
    if (B.route != 1) return;   // direct-route band: written by k_direct_reduce
    if constexpr (sizeof(T) == 4 && !XI) {
        const C v = gather_node_f32<MW>(ntab[i], i - B.node_off, B, bands, grid, cheb32, q, kb_b, fpp);
        f[j] = rmul ? cmulc(rmul[j], v) : v;
        return;
    }
    const double2 wv = ws[i];
    const double xs = XI ? 0.5 * wv.x : wv.x;
    const double x = xs - floor(xs);
    C acc = {(T)0, (T)0};
    const double t0 = (double)B.n * x;
    const double u = floor(t0);
    const T fr = (T)(t0 - u);
    const int64_t lo = (int64_t)u - (MW - 1);
    T phi[2 * MW];
    const T kb = XI ? kb_b : (T)B.kb;   // the window shape of the band's grids
#pragma unroll
    for (int t = 0; t < 2 * MW; ++t) phi[t] = kb_window<T>(fr + (T)(MW - 1 - t), (T)MW, kb);
    const int64_t nmask = B.n - 1;
    const C* g = grid + B.grid_off;
    if constexpr (sizeof(T) == 8 && !XI) {
        if (B.nsub > 0) {   // split band (FP64): its sub-bands' grids, each with its centre phase
            T Ls[kMaxQ];
            if (B.nrhs > 1) bary_weights<T>(kTwoPiD * wv.y, B, q, cheb, Ls);
            else Ls[0] = (T)1;   // the Y_M band: one right-hand side
            for (int sb = 0; sb < B.nsub; ++sb) {
                const BandDev S = bands[B.sub0 + sb];
                const C* gs = grid + S.grid_off;
                C a = {(T)0, (T)0};
                for (int s = 0; s < S.nrhs; ++s) {
                    const C v = tap_sum<MW>(gs + (int64_t)s * S.n, lo, nmask, phi);
                    a.x += Ls[s] * v.x;
                    a.y += Ls[s] * v.y;
                }
                const double ph = frac_turns((double)(S.k0 + (S.Nm >> 1)), x);
                acc = cadd(acc, cmul(a, expipi<T>((T)(2.0 * ph))));
            }
            f[j] = rmul ? cmulc(rmul[j], acc) : acc;
            return;
        }
    }
    if constexpr (sizeof(T) == 4) {   // XI (real exponents) in FP32
        if (B.nrhs > 1) {
            const double tau = (kTwoPiD * wv.y - B.yc) * B.yh_inv;
            const float th = (float)tau, tl = (float)(tau - (double)th);
            acc = gather_rhs_f32<MW>(g, B, lo, nmask, phi, th, tl, q, cheb32);
        } else {
            acc = tap_sum<MW>(g, lo, nmask, phi);
        }
    } else if (B.nrhs == 1) {
        acc = tap_sum<MW>(g, lo, nmask, phi);
    } else if constexpr (sizeof(T) == 8) {
        T Ls[kMaxQ];
        bary_weights<T>(kTwoPiD * wv.y, B, q, cheb, Ls);
        for (int s = 0; s < q; ++s) {
            const C a = tap_sum<MW>(g + (int64_t)s * B.n, lo, nmask, phi);
            acc.x += Ls[s] * a.x;
            acc.y += Ls[s] * a.y;
        }
    }
    C val;
    if constexpr (XI) {
        // exp(2 pi i xc x) / Phi(x/2), x = Re w in [-1/2, 1/2]
        const double ph = frac_turns(B.xc, wv.x);
        const T v = (T)(kTwoPiD * 0.5 * wv.x);
        const T arg = kb_b * kb_b - v * v;
        const T r = (T)MW * sqrt(arg > (T)0 ? arg : (T)0);
        T i0;
        if constexpr (sizeof(T) == 4) i0 = cyl_bessel_i0f(r);
        else i0 = cyl_bessel_i0(r);
        const T iphi = (T)1 / ((T)kPi * i0);
        const C e = expipi<T>((T)(2.0 * ph));
        val = cmul(acc, C{e.x * iphi, e.y * iphi});
    } else {
        // centring shift exp(2 pi i (N_m/2) x)
        double ph = (double)(B.Nm >> 1) * x;   // N_m a power of two: exact
        ph -= floor(ph);
        if (ph >= 0.5) ph -= 1.0;
        val = cmul(acc, expipi<T>((T)(2.0 * ph)));
    }
    f[j] = rmul ? cmulc(rmul[j], val) : val;
}

// ---------------------------------------------------------------------------
// Adjoint: spread (transpose of the gather), FFT with sign -, combine.

// The float-pair form's spreading preparation: k_spread_prep's per-node
// window taps, barycentric weights and shifted r_j in pairs (the window from
// one pair exponential, the weights as in k_gather_ff); the phase (N_m/2) x
// mod 1 is reduced exactly in double.
template <int MW>
__global__ void __launch_bounds__(256) k_spread_prep_ff(int64_t M, const double2* __restrict__ ws,
                                                        const int32_t* __restrict__ perm,
                                                        const int32_t* __restrict__ bandid,
                                                        const BandDev* __restrict__ bands,
                                                        const double2* __restrict__ r,
                                                        const float* __restrict__ cheb32, int q,
                                                        ff* __restrict__ sp_phi, ff* __restrict__ sp_L,
                                                        ffc* __restrict__ sp_rv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const BandDev B = bands[bandid[i]];
    if (B.route != 1) return;
    const double2 wv = ws[i];
    const double x = wv.x - floor(wv.x);
    const double t0 = (double)B.n * x;
    const ff fr = ff(t0 - floor(t0));
    double ph = (double)(B.Nm >> 1) * x;   // N_m a power of two: exact
    ph -= floor(ph);
    if (ph >= 0.5) ph -= 1.0;
    ffc e;
    ff_sincospi(ff(2.0 * ph), &e.y, &e.x);
    const double2 rj = r[perm[i]];
    sp_rv[i] = cmulc(ffc{ff(rj.x), ff(rj.y)}, e);
    const ff kb = ff(B.kb);
#pragma unroll
    for (int t = 0; t < 2 * MW; ++t) sp_phi[i * (2 * MW) + t] = ff_kb_window(fr + ff(MW - 1 - t), (float)MW, kb);
    if (B.nrhs > 1) {
        const ff tf = ff((kTwoPiD * wv.y - B.yc) * B.yh_inv);
        ff L[kMaxQ];
        ff den = ff(0);
        int hit = -1;
        for (int s = 0; s < q; ++s) {
            const ff d = tf - ff(cheb32[s], cheb32[q + s]);
            if (d.hi == 0.f && d.lo == 0.f) {
                hit = s;
                L[s] = ff(0);
                continue;
            }
            L[s] = ff_div(ff(cheb32[2 * q + s], cheb32[3 * q + s]), d);
            den += L[s];
        }
        for (int s = 0; s < q; ++s)
            sp_L[i * q + s] = hit >= 0 ? (s == hit ? ff(1) : ff(0)) : ff_div(L[s], den);
    }
}

// Adjoint spreading, the transpose of the gather, without atomics in two
// steps.  k_spread_prep: for every sorted node of an NFFT band its 2 m_w window
// taps, its barycentric weights L_s(y_j) and rv_j = r_j exp(-2 pi i (N_m/2) x_j).
// XI (real exponents): taps at x_j/2 and rv_j = r_j exp(-2 pi i xc x_j) /
// Phi(x_j/2), the conjugate of the forward epilogue.
template <typename T, int MW, bool XI = false>
__global__ void __launch_bounds__(256) k_spread_prep(int64_t M, const double2* __restrict__ ws,
                                                     const int32_t* __restrict__ perm,
                                                     const int32_t* __restrict__ bandid,
                                                     const BandDev* __restrict__ bands,
                                                     const C_t<T>* __restrict__ r,
                                                     const double* __restrict__ cheb, int q, T kb_b,
                                                     T* __restrict__ sp_phi, T* __restrict__ sp_L,
                                                     C_t<T>* __restrict__ sp_rv) {
    using C = C_t<T>;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const BandDev B = bands[bandid[i]];
    if (B.route != 1) return;
    const double2 wv = ws[i];
    const double xs = XI ? 0.5 * wv.x : wv.x;
    const double x = xs - floor(xs);
    const double t0 = (double)B.n * x;
    const T fr = (T)(t0 - floor(t0));
    if (B.nsub > 0) {   // split band: each sub-band applies its own centre phase
        sp_rv[i] = r[perm[i]];
    } else if constexpr (XI) {
        const double ph = frac_turns(B.xc, wv.x);
        const T v = (T)(kTwoPiD * 0.5 * wv.x);
        const T arg = kb_b * kb_b - v * v;
        const T rr = (T)MW * sqrt(arg > (T)0 ? arg : (T)0);
        T i0;
        if constexpr (sizeof(T) == 4) i0 = cyl_bessel_i0f(rr);
        else i0 = cyl_bessel_i0(rr);
        const C rv = cmulc(r[perm[i]], expipi<T>((T)(2.0 * ph)));
        sp_rv[i] = cscale(rv, (T)1 / ((T)kPi * i0));
    } else {
        double ph = (double)(B.Nm >> 1) * x;   // N_m a power of two: exact
        ph -= floor(ph);
        if (ph >= 0.5) ph -= 1.0;
        sp_rv[i] = cmulc(r[perm[i]], expipi<T>((T)(2.0 * ph)));
    }
    const T kb = XI ? kb_b : (T)B.kb;   // the window shape of the band's grid
#pragma unroll
    for (int t = 0; t < 2 * MW; ++t)
        sp_phi[i * (2 * MW) + t] = kb_window<T>(fr + (T)(MW - 1 - t), (T)MW, kb);
    if (B.nrhs > 1) {
        T Ls[kMaxQ];
        bary_weights<T>(kTwoPiD * wv.y, B, q, cheb, Ls);
        for (int s = 0; s < q; ++s) sp_L[i * q + s] = Ls[s];
    }
}

// First sorted node of [lo, hi) whose cell is >= v (cells ascend within a band).
__device__ __forceinline__ int64_t lower_cell(const int32_t* __restrict__ cell, int64_t lo,
                                              int64_t hi, int64_t v) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cell[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Sum over the nodes that cover grid cell l of one NFFT band: the nodes whose
// cell u lies in [l - m_w, l + m_w - 1] (mod n) form a contiguous range of the
// band's cell-sorted nodes (two near the ends); node j adds window tap
// t = l - u + m_w - 1 times rv_j, times L_s(y_j) for right-hand side s.  The
// lanes lane, lane + stride, ... of the range are summed into acc.
template <typename T, int MW>
__device__ __forceinline__ void spread_cell_sum(const BandDev& B, int64_t l,
                                                const int32_t* __restrict__ cell,
                                                const T* __restrict__ sp_phi,
                                                const T* __restrict__ sp_L,
                                                const C_t<T>* __restrict__ sp_rv,
                                                const double2* __restrict__ ws, int q,
                                                int lane, int stride, C_t<T>* acc) {
    using C = C_t<T>;
    // a sub-band: node j's value carries exp(-2 pi i kc x_j), kc its centre
    const double kc = (double)(B.k0 + (B.Nm >> 1));
    const int64_t n = B.n, nb0 = B.node_off, nend = B.node_off + B.nodes;
    int64_t ra[2][2];
    int nrange = 0;
    const int64_t c0 = l - MW, c1 = l + MW - 1;
    if (c0 < 0) {
        ra[0][0] = n + c0; ra[0][1] = n - 1;
        ra[1][0] = 0; ra[1][1] = c1;
        nrange = 2;
    } else if (c1 >= n) {
        ra[0][0] = c0; ra[0][1] = n - 1;
        ra[1][0] = 0; ra[1][1] = c1 - n;
        nrange = 2;
    } else {
        ra[0][0] = c0; ra[0][1] = c1;
        nrange = 1;
    }
    const int nr = B.nrhs;
    for (int rr = 0; rr < nrange; ++rr) {
        const int64_t j0 = lower_cell(cell, nb0, nend, ra[rr][0]);
        const int64_t j1 = lower_cell(cell, j0, nend, ra[rr][1] + 1);
        for (int64_t j = j0 + lane; j < j1; j += stride) {
            int64_t t = (l - cell[j] + MW - 1) % n;
            if (t < 0) t += n;
            C w = cscale(sp_rv[j], sp_phi[j * (2 * MW) + t]);
            if constexpr (!std::is_same<T, ff>::value) {   // (no sub-bands in float pairs)
                if (B.parent >= 0) {
                    const double xj = ws[j].x - floor(ws[j].x);
                    w = cmul(w, expipi<T>((T)(-2.0 * frac_turns(kc, xj))));
                }
            }
            if (nr == 1) {
                acc[0] = cadd(acc[0], w);
            } else {
                for (int s = 0; s < nr; ++s) {
                    const T L = sp_L[j * q + s];
                    acc[s].x += L * w.x;
                    acc[s].y += L * w.y;
                }
            }
        }
    }
}

__device__ __forceinline__ int find_cell_band(const Plan::CellBand* __restrict__ cbs, int ncb,
                                              int64_t g) {
    int lo = 0, hi = ncb;   // last entry with prefix <= g
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cbs[mid].prefix <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

// A spread grid value as stored: C_t<T>, or rounded to a float pair (the grids
// of the float-pair form, whose spreading runs in double).
template <typename G, typename C> __device__ __forceinline__ G grid_value(const C& v) {
    if constexpr (std::is_same<G, ffc>::value) return ffc{ff(v.x), ff(v.y)};
    else return v;
}

// k_spread_cells: one thread per (sparse NFFT band, grid cell l); writes a_s[l]
// for every right-hand side s.
template <typename T, int MW, typename G = C_t<T>>
__global__ void __launch_bounds__(256) k_spread_cells(int ncb, const Plan::CellBand* __restrict__ cbs,
                                                      int64_t total, const BandDev* __restrict__ bands,
                                                      const int32_t* __restrict__ cell,
                                                      const T* __restrict__ sp_phi,
                                                      const T* __restrict__ sp_L,
                                                      const C_t<T>* __restrict__ sp_rv,
                                                      const double2* __restrict__ ws, int q,
                                                      G* __restrict__ grid) {
    using C = C_t<T>;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int cb = find_cell_band(cbs, ncb, g);
    const BandDev B = bands[cbs[cb].band];
    const int64_t l = g - cbs[cb].prefix;
    C acc[kMaxQ];
    for (int s = 0; s < B.nrhs; ++s) acc[s] = C{(T)0, (T)0};
    spread_cell_sum<T, MW>(B, l, cell, sp_phi, sp_L, sp_rv, ws, q, 0, 1, acc);
    G* gb = grid + B.grid_off + l;
    for (int s = 0; s < B.nrhs; ++s) gb[(int64_t)s * B.n] = grid_value<G>(acc[s]);
}

__device__ __forceinline__ float shfl_xor_t(float v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ double shfl_xor_t(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ ff shfl_xor_t(ff v, int off) {
    return ff(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}

// Dense NFFT bands (many nodes per cell): one CTA of kSpreadDense threads per
// cell, threads strided over the covering nodes; the thread sums are combined
// in a fixed order (a shuffle tree per warp, then the warps in order).
constexpr int kSpreadDense = 256;

template <typename T, int MW, typename G = C_t<T>>
__global__ void __launch_bounds__(kSpreadDense) k_spread_cells_warp(int ncb, const Plan::CellBand* __restrict__ cbs,
                                                                    int64_t total,
                                                                    const BandDev* __restrict__ bands,
                                                                    const int32_t* __restrict__ cell,
                                                                    const T* __restrict__ sp_phi,
                                                                    const T* __restrict__ sp_L,
                                                                    const C_t<T>* __restrict__ sp_rv,
                                                                    const double2* __restrict__ ws, int q,
                                                                    G* __restrict__ grid) {
    using C = C_t<T>;
    __shared__ C red[kSpreadDense / 32][kMaxQ];
    const int64_t g = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (g >= total) return;
    const int cb = find_cell_band(cbs, ncb, g);
    const BandDev B = bands[cbs[cb].band];
    const int64_t l = g - cbs[cb].prefix;
    C acc[kMaxQ];
    for (int s = 0; s < B.nrhs; ++s) acc[s] = C{(T)0, (T)0};
    spread_cell_sum<T, MW>(B, l, cell, sp_phi, sp_L, sp_rv, ws, q, threadIdx.x, kSpreadDense, acc);
    for (int s = 0; s < B.nrhs; ++s) {
        T x = acc[s].x, y = acc[s].y;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            x += shfl_xor_t(x, off);
            y += shfl_xor_t(y, off);
        }
        if (lane == 0) red[w][s] = C{x, y};
    }
    __syncthreads();
    const int s = threadIdx.x;
    if (s < B.nrhs) {
        C sum = red[0][s];
        for (int ww = 1; ww < kSpreadDense / 32; ++ww) sum = cadd(sum, red[ww][s]);
        grid[B.grid_off + l + (int64_t)s * B.n] = grid_value<G>(sum);
    }
}

// Sum of r over the Z^0 nodes (the first z0 sorted nodes): c_out[0] gets it.
template <typename T>
__global__ void k_z0_sum(int64_t z0, const int32_t* __restrict__ perm,
                         const C_t<T>* __restrict__ r, C_t<T>* __restrict__ out) {
    __shared__ T sx[256], sy[256];
    T ax = 0, ay = 0;
    for (int64_t i = threadIdx.x; i < z0; i += 256) {
        const C_t<T> v = r[perm[i]];
        ax += v.x;
        ay += v.y;
    }
    sx[threadIdx.x] = ax;
    sy[threadIdx.x] = ay;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sx[threadIdx.x] += sx[threadIdx.x + h];
            sy[threadIdx.x] += sy[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = C_t<T>{sx[0], sy[0]};
}

// c_out[k] = [k == 0] z0sum + sum_bands sum_s D[s][k] b_s[(k - N_m/2) mod n],
// accumulated in T (double for the float-pair form, whose grids G and weights
// DT are float pairs).
template <typename T, typename G = C_t<T>, typename DT = T>
__global__ void k_combine(int64_t N, int levels, const BandDev* __restrict__ bands,
                          const DT* __restrict__ D, const G* __restrict__ grid,
                          const C_t<T>* __restrict__ z0sum, const C_t<T>* __restrict__ cdir,
                          C_t<T>* __restrict__ cout) {
    using C = C_t<T>;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    C acc = (k == 0) ? *z0sum : C{(T)0, (T)0};
    if (cdir) acc = cadd(acc, cdir[k]);
    for (int b = 1; b <= levels; ++b) {
        BandDev B = bands[b];
        if (B.route != 1 || k >= B.K) continue;
        for (int c = 0; c < B.nsub; ++c) {   // split band: the sub-band holding k
            const BandDev S = bands[B.sub0 + c];
            if (k >= S.k0 && k < S.k0 + S.K) {
                B = S;
                break;
            }
        }
        const int64_t kl = k - B.k0;   // frequency within the (sub-)band
        const int64_t i = (kl - (B.Nm >> 1)) & (B.n - 1);
        const DT* Dk = D + B.D_off + kl;
        const G* g = grid + B.grid_off + i;
        for (int s = 0; s < B.nrhs; ++s) {
            const T d = (T)Dk[(int64_t)s * B.K];
            const G v = g[(int64_t)s * B.n];
            acc.x += d * (T)v.x;
            acc.y += d * (T)v.y;
        }
    }
    cout[k] = acc;
}

// ---------------------------------------------------------------------------
// Orchestration.

static void large_split(int log2n, int* l1, int* l2) {
    *l1 = (log2n + 1) / 2;
    *l2 = log2n / 2;
}

template <typename T, int SIGN, int MODE, bool DERIV>
static cudaError_t fft_bands(Plan& p, const void* c, cudaStream_t st) {
    using C = C_t<T>;
    C* grid = (C*)p.d_grid;
    cudaError_t e = cudaSuccess;
    if (!p.small_work.empty()) {
        double bytes = 0;
        for (const SmallWork& w : p.small_work) {
            const BandDev& B = p.bands[w.band].dev;
            bytes += (double)w.nfft * (B.n * sizeof(C) * (MODE == 0 ? 1 : 2) +
                                       (MODE == 0 ? B.K * (sizeof(C) + sizeof(T)) : 0));
        }
        int slot;
        timer_begin(p, "small_fft", bytes, st, &slot);
        e = launch_small_fft<T, SIGN, MODE, DERIV>(p.d_small, (int)p.small_work.size(), p.d_bands,
                                                   (const C*)c, (const T*)p.d_D, grid,
                                                   (const C*)p.d_tw, st);
        timer_end(p, slot, st);
        ++p.launches;
        if (e != cudaSuccess) return e;
    }
    for (const PassGroup& g : p.pass_groups) {
        int l1, l2;
        large_split(g.log2n, &l1, &l2);
        const int64_t n = (int64_t)1 << g.log2n;
        double kbytes = 0;   // forward input reads: c and D over the items' K
        for (int i = 0; i < g.count; ++i) kbytes += (double)p.bands[p.pass_items[g.start + i].band].dev.K;
        const double b1 = (double)g.count * n * sizeof(C) +
                          (MODE == 0 ? kbytes * (sizeof(C) + sizeof(T)) : (double)g.count * n * sizeof(C));
        double b2 = 0;   // Y read + grid write, or Y read + entries + partials (fused)
        for (int i = 0; i < g.count; ++i) {
            const BandHost& bh = p.bands[p.pass_items[g.start + i].band];
            if (SIGN > 0 && MODE == 0 && bh.dev.fused) {   // Y read; entries read, partials written
                const int NQ = (pass_tiles(8, (g.log2n + 1) / 2, FL_P2_THREADS_F32) + 3) / 4;
                b2 += (double)n * sizeof(C) + (double)bh.fentries * (8.0 + 16.0 * NQ + 8.0);
            } else {
                b2 += 2.0 * n * sizeof(C);
            }
        }
        int slot;
        timer_begin(p, "fft_pass1", b1, st, &slot);
        e = launch_pass1<T, SIGN, MODE, DERIV>(p.d_pass + g.start, g.count, p.d_bands, l1, l2,
                                               (const C*)c, (const T*)p.d_D, grid, (C*)p.d_Y,
                                               (const C*)p.d_tw, st);
        timer_end(p, slot, st);
        if (e != cudaSuccess) return e;
        timer_begin(p, "fft_pass2", b2, st, &slot);
        e = launch_pass2<T, SIGN>(p.d_pass + g.start, g.count, p.d_bands, l1, l2, (const C*)p.d_Y,
                                  grid, (const C*)p.d_tw,
                                  FuseArgs{p.d_frbs, p.d_fent, p.d_fphi, p.d_fpp}, st);
        timer_end(p, slot, st);
        p.launches += 2;
        if (e != cudaSuccess) return e;
    }
    return e;
}

template <typename T, int MW>
static cudaError_t gather_t(Plan& p, const void* c, void* f, bool deriv, const void* rmul,
                            cudaStream_t st) {
    if (p.xi_mode) {
        int slot;
        timer_begin(p, "gather", 0.0, st, &slot);
        k_gather<T, MW, true><<<(unsigned)((p.M + 255) / 256), 256, 0, st>>>(
            p.M, p.d_ws, p.d_perm, p.d_bandid, p.d_bands, (const C_t<T>*)p.d_grid, p.d_cheb,
            p.d_cheb32, p.q, (T)p.kb_b, (const C_t<T>*)c, 0, nullptr, nullptr, nullptr, (C_t<T>*)f);
        timer_end(p, slot, st);
        ++p.launches;
        return cudaGetLastError();
    }
    using C = C_t<T>;
    double bytes = (double)p.M * (sizeof(double2) + 4 + 1 + sizeof(C));
    for (int b = 1; b < (int)p.bands.size(); ++b) {
        const BandDev& B = p.bands[b].dev;
        if (B.route != 1 || B.nsub > 0) continue;
        if (B.fused) {
            bytes += (double)p.bands[b].nodes * B.nrhs * B.pparts * sizeof(C);
            continue;
        }
        bytes += std::min<double>((double)B.nrhs * B.n * sizeof(C),
                                  (double)p.bands[b].nodes * B.nrhs * 2 * MW * sizeof(C));
    }
    int slot;
    timer_begin(p, "gather", bytes, st, &slot);
    k_gather<T, MW><<<(unsigned)((p.M + 255) / 256), 256, 0, st>>>(
        p.M, p.d_ws, p.d_perm, p.d_bandid, p.d_bands, (const C*)p.d_grid, p.d_cheb, p.d_cheb32,
        p.q, (T)p.kb_b, (const C*)c, deriv ? 1 : 0, (const C*)rmul, p.d_fpp, p.d_ntab, (C*)f);
    timer_end(p, slot, st);
    ++p.launches;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t gather_dispatch(Plan& p, const void* c, void* f, bool deriv, const void* rmul,
                                   cudaStream_t st) {
    switch (p.mw) {
#define FL_MW_CASE(W) \
    case W: return gather_t<T, W>(p, c, f, deriv, rmul, st);
        FL_MW_CASE(2) FL_MW_CASE(3) FL_MW_CASE(4) FL_MW_CASE(5) FL_MW_CASE(6) FL_MW_CASE(7)
        FL_MW_CASE(8) FL_MW_CASE(9) FL_MW_CASE(10) FL_MW_CASE(11) FL_MW_CASE(12)
#undef FL_MW_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
static cudaError_t forward_t(Plan& p, const void* c, void* f, bool deriv, const void* rmul,
                             cudaStream_t st) {
    if (p.M == 0) return cudaSuccess;
    cudaError_t e = deriv ? fft_bands<T, +1, 0, true>(p, c, st) : fft_bands<T, +1, 0, false>(p, c, st);
    if (e != cudaSuccess) return e;
    if ((e = run_direct_forward(p, c, f, deriv, rmul, st)) != cudaSuccess) return e;
    return gather_dispatch<T>(p, c, f, deriv, rmul, st);
}

// Real exponents: frequency spreading of every band, the FFTs of the grids
// (inputs read from the grids, sign +), and the gather at x/2 with the NNFFT
// epilogue.
template <typename T>
static cudaError_t forward_xi_t(Plan& p, const void* c, void* f, cudaStream_t st) {
    cudaError_t e = launch_xi_spread(p, c, st);
    if (e != cudaSuccess) return e;
    e = fft_bands<T, 1, 1, false>(p, nullptr, st);
    if (e != cudaSuccess) return e;
    return gather_dispatch<T>(p, c, f, false, nullptr, st);
}

cudaError_t run_forward_xi(Plan& p, const void* c, void* f, cudaStream_t st) {
    return p.prec == FL_FP64 ? forward_xi_t<double>(p, c, f, st) : forward_xi_t<float>(p, c, f, st);
}

// FP64-accuracy form in float pairs: c converted once to pairs; the FFTs of
// the band grids, the direct bands and the gather (window, barycentric
// weights, shift) in float pairs, with the phases reduced exactly in double.
// (deriv: the k-weighted coefficients 2 pi i k c_k, formed in double and then
// rounded to pairs)
__global__ void k_to_ff(int64_t n, const double2* __restrict__ in, int deriv, ffc* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v = in[i];
    if (deriv) {
        const double w = kTwoPiD * (double)i;
        v = double2{-w * v.y, w * v.x};
    }
    out[i] = ffc{ff(v.x), ff(v.y)};
}

// The gather of the float-pair form: k_gather's steps with the window values,
// tap sums, barycentric weights and recombination in float pairs (fl_ffmath.cuh)
// instead of double; the phases n x mod 1 and (N_m/2) x mod 1 and tau are
// still reduced exactly in double (once per node).  The barycentric sum is
// accumulated in one pass, sum_s L_s a_s / sum_s L_s with L_s = lambda_s /
// (tau - t_s); an exact hit tau = t_s returns a_s.
template <int MW>
__global__ void __launch_bounds__(256) k_gather_ff(int64_t M, const double2* __restrict__ ws,
                                                   const int32_t* __restrict__ perm,
                                                   const int32_t* __restrict__ bandid,
                                                   const BandDev* __restrict__ bands,
                                                   const ffc* __restrict__ grid,
                                                   const float* __restrict__ cheb32, int q,
                                                   double kb_b, const double2* __restrict__ c,
                                                   int deriv, const double2* __restrict__ rmul,
                                                   double2* __restrict__ f) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int b = bandid[i];
    const int32_t j = perm[i];
    const BandDev B = bands[b];
    if (B.K == 0 && B.n == 0) {   // Z^0: c_0 (its k-weighted term is 0)
        f[j] = (deriv || rmul) ? double2{0.0, 0.0} : c[B.c_off];
        return;
    }
    if (B.route != 1) return;     // direct-route band: written by the direct kernels
    const double2 wv = ws[i];
    const double x = wv.x - floor(wv.x);
    const double t0 = (double)B.n * x;
    const double u = floor(t0);
    const ff fr = ff(t0 - u);
    const int64_t lo = (int64_t)u - (MW - 1);
    const ff bb = ff(kb_b);
    ff phi[2 * MW];
#pragma unroll
    for (int t = 0; t < 2 * MW; ++t) phi[t] = ff_kb_window(fr + ff(MW - 1 - t), (float)MW, bb);
    const int64_t nmask = B.n - 1;
    const ffc* g = grid + B.grid_off;
    ffc acc;
    if (B.nrhs == 1) {
        acc = tap_sum<MW>(g, lo, nmask, phi);
    } else {
        const ff tf = ff((kTwoPiD * wv.y - B.yc) * B.yh_inv);
        ff den = ff(0);
        ffc num = {ff(0), ff(0)}, ahit = {ff(0), ff(0)};
        bool hit = false;
        for (int s = 0; s < q; ++s) {
            const ffc a = tap_sum<MW>(g + (int64_t)s * B.n, lo, nmask, phi);
            const ff d = tf - ff(cheb32[s], cheb32[q + s]);
            if (d.hi == 0.f && d.lo == 0.f) {
                hit = true;
                ahit = a;
                continue;
            }
            const ff L = ff_div(ff(cheb32[2 * q + s], cheb32[3 * q + s]), d);
            den += L;
            num.x += L * a.x;
            num.y += L * a.y;
        }
        acc = hit ? ahit : ffc{ff_div(num.x, den), ff_div(num.y, den)};
    }
    // centring shift exp(2 pi i (N_m/2) x); N_m is a power of two, so the
    // product is exact in double
    double ph = (double)(B.Nm >> 1) * x;
    ph -= floor(ph);
    if (ph >= 0.5) ph -= 1.0;
    ffc e;
    ff_sincospi(ff(2.0 * ph), &e.y, &e.x);
    const ffc v = cmul(acc, e);
    const double2 out = double2{(double)v.x, (double)v.y};
    // with rmul: rmul[j] conj(f'_j) (node gradient, see fl_grad_w)
    f[j] = rmul ? cmulc(rmul[j], out) : out;
}

template <int MW>
static cudaError_t gather_ff_t(Plan& p, const void* c, void* f, bool deriv, const void* rmul,
                               cudaStream_t st) {
    double bytes = (double)p.M * (sizeof(double2) + 4 + 1 + sizeof(double2));
    for (int b = 1; b <= p.levels; ++b) {
        const BandDev& B = p.bands[b].dev;
        if (B.route != 1) continue;
        bytes += std::min<double>((double)B.nrhs * B.n * sizeof(ffc),
                                  (double)p.bands[b].nodes * B.nrhs * 2 * MW * sizeof(ffc));
    }
    int slot;
    timer_begin(p, "gather", bytes, st, &slot);
    k_gather_ff<MW><<<(unsigned)((p.M + 255) / 256), 256, 0, st>>>(
        p.M, p.d_ws, p.d_perm, p.d_bandid, p.d_bands, (const ffc*)p.d_grid, p.d_cheb32, p.q,
        p.kb_b, (const double2*)c, deriv ? 1 : 0, (const double2*)rmul, (double2*)f);
    timer_end(p, slot, st);
    ++p.launches;
    return cudaGetLastError();
}

// (deriv: Algorithm 2 on the k-weighted coefficients, the derivative in w;
// rmul: the node gradient rmul_j conj(f'_j))
static cudaError_t forward_ff(Plan& p, const void* c, void* f, bool deriv, const void* rmul,
                              cudaStream_t st) {
    if (p.M == 0) return cudaSuccess;
    k_to_ff<<<(unsigned)((p.N + 255) / 256), 256, 0, st>>>(p.N, (const double2*)c, deriv ? 1 : 0,
                                                           (ffc*)p.d_cff);
    ++p.launches;
    cudaError_t e = fft_bands<ff, +1, 0, false>(p, p.d_cff, st);
    if (e != cudaSuccess) return e;
    if ((e = run_direct_forward(p, c, f, deriv, rmul, st)) != cudaSuccess) return e;
    switch (p.mw) {
#define FL_MW_CASE(W) \
    case W: return gather_ff_t<W>(p, c, f, deriv, rmul, st);
        FL_MW_CASE(2) FL_MW_CASE(3) FL_MW_CASE(4) FL_MW_CASE(5) FL_MW_CASE(6) FL_MW_CASE(7)
        FL_MW_CASE(8) FL_MW_CASE(9) FL_MW_CASE(10) FL_MW_CASE(11) FL_MW_CASE(12)
#undef FL_MW_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t run_forward(Plan& p, const void* c, void* f, bool deriv, cudaStream_t st,
                        const void* rmul) {
    if (p.prec == FL_FP64_FF) return forward_ff(p, c, f, deriv, rmul, st);
    return p.prec == FL_FP64 ? forward_t<double>(p, c, f, deriv, rmul, st)
                             : forward_t<float>(p, c, f, deriv, rmul, st);
}

template <typename T, int MW, typename G = C_t<T>>
static cudaError_t spread_t(Plan& p, const void* r, cudaStream_t st) {
    using C = C_t<T>;
    if (p.cell_bands.empty()) return cudaSuccess;
    int slot;
    timer_begin(p, "spread", 0.0, st, &slot);
    if constexpr (std::is_same<T, ff>::value) {
        k_spread_prep_ff<MW><<<(unsigned)((p.M + 255) / 256), 256, 0, st>>>(
            p.M, p.d_ws, p.d_perm, p.d_bandid, p.d_bands, (const double2*)r, p.d_cheb32, p.q,
            (ff*)p.d_sp_phi, (ff*)p.d_sp_L, (ffc*)p.d_sp_rv);
    } else {
        auto prep = p.xi_mode ? k_spread_prep<T, MW, true> : k_spread_prep<T, MW, false>;
        prep<<<(unsigned)((p.M + 255) / 256), 256, 0, st>>>(
            p.M, p.d_ws, p.d_perm, p.d_bandid, p.d_bands, (const C*)r, p.d_cheb, p.q, (T)p.kb_b,
            (T*)p.d_sp_phi, (T*)p.d_sp_L, (C*)p.d_sp_rv);
    }
    if (p.cells_total > 0)
        k_spread_cells<T, MW, G><<<(unsigned)((p.cells_total + 255) / 256), 256, 0, st>>>(
            (int)p.n_sparse_cb, p.d_cell_bands, p.cells_total, p.d_bands, p.d_cell,
            (const T*)p.d_sp_phi, (const T*)p.d_sp_L, (const C*)p.d_sp_rv, p.d_ws, p.q, (G*)p.d_grid);
    if (p.cells_dense > 0)
        k_spread_cells_warp<T, MW, G><<<(unsigned)p.cells_dense, kSpreadDense, 0, st>>>(
            (int)(p.cell_bands.size() - p.n_sparse_cb), p.d_cell_bands + p.n_sparse_cb,
            p.cells_dense, p.d_bands, p.d_cell, (const T*)p.d_sp_phi, (const T*)p.d_sp_L,
            (const C*)p.d_sp_rv, p.d_ws, p.q, (G*)p.d_grid);
    timer_end(p, slot, st);
    p.launches += 1 + (p.cells_total > 0) + (p.cells_dense > 0);
    return cudaGetLastError();
}

// T: the arithmetic of the direct bands and the combine; FT: that of the
// spreading and the FFTs (T, or float pairs ff with T = double for the
// float-pair form, whose combine reads pair grids and weights in double).
template <typename T, typename FT = T>
static cudaError_t adjoint_t(Plan& p, const void* r, void* cout, cudaStream_t st) {
    using C = C_t<T>;
    using G = C_t<FT>;
    cudaError_t e;
    switch (p.mw) {
#define FL_MW_CASE(W) \
    case W: e = spread_t<FT, W, G>(p, r, st); break;
        FL_MW_CASE(2) FL_MW_CASE(3) FL_MW_CASE(4) FL_MW_CASE(5) FL_MW_CASE(6) FL_MW_CASE(7)
        FL_MW_CASE(8) FL_MW_CASE(9) FL_MW_CASE(10) FL_MW_CASE(11) FL_MW_CASE(12)
#undef FL_MW_CASE
        default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if ((e = fft_bands<FT, -1, 1, false>(p, nullptr, st)) != cudaSuccess) return e;
    if (p.xi_mode) return launch_xi_combine(p, cout, st);   // no direct bands, Z^0 adds 0
    if ((e = run_direct_adjoint(p, r, st)) != cudaSuccess) return e;
    C* z0sum = (C*)p.d_z0;
    k_z0_sum<T><<<1, 256, 0, st>>>(p.z0_nodes, p.d_perm, (const C*)r, z0sum);
    int slot;
    timer_begin(p, "combine", 0.0, st, &slot);
    k_combine<T, G, FT><<<(unsigned)((p.N + 255) / 256), 256, 0, st>>>(
        p.N, p.levels, p.d_bands, (const FT*)p.d_D, (const G*)p.d_grid, z0sum,
        p.direct_ranges.empty() ? nullptr : (const C*)p.d_cdir, (C*)cout);
    timer_end(p, slot, st);
    p.launches += 2;
    return cudaGetLastError();
}

cudaError_t run_adjoint(Plan& p, const void* r, void* cout, cudaStream_t st) {
    if (p.prec == FL_FP64_FF) return adjoint_t<double, ff>(p, r, cout, st);
    return p.prec == FL_FP64 ? adjoint_t<double>(p, r, cout, st) : adjoint_t<float>(p, r, cout, st);
}

// out[i] = conj(in[i]) (in == out allowed)
template <typename T>
__global__ void k_conj(int64_t n, const C_t<T>* in, C_t<T>* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const C_t<T> v = in[i];
        out[i] = C_t<T>{v.x, -v.y};
    }
}

template <typename T, typename FT = T>
static cudaError_t transposed_t(Plan& p, const void* g, void* out, cudaStream_t st) {
    using C = C_t<T>;
    if (p.M > 0) {
        if (!p.d_stage_r) {
            cudaError_t e = cudaMalloc(&p.d_stage_r, (size_t)p.M * sizeof(C));
            if (e != cudaSuccess) return e;
        }
        k_conj<T><<<(unsigned)((p.M + 255) / 256), 256, 0, st>>>(p.M, (const C*)g, (C*)p.d_stage_r);
        ++p.launches;
    }
    cudaError_t e = adjoint_t<T, FT>(p, p.M > 0 ? p.d_stage_r : g, out, st);
    if (e != cudaSuccess) return e;
    k_conj<T><<<(unsigned)((p.N + 255) / 256), 256, 0, st>>>(p.N, (const C*)out, (C*)out);
    ++p.launches;
    return cudaGetLastError();
}

// g_k = sum_j ghat_j z_j^k, k = 0..N-1 (C^T ghat = conj(C^* conj(ghat))).
cudaError_t run_transposed(Plan& p, const void* g, void* out, cudaStream_t st) {
    if (p.prec == FL_FP64_FF) return transposed_t<double, ff>(p, g, out, st);
    return p.prec == FL_FP64 ? transposed_t<double>(p, g, out, st) : transposed_t<float>(p, g, out, st);
}

}  // namespace fl
