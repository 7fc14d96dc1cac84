// fl_xi.cu -- real exponents: f_j = sum_k c_k z_j^{xi_k}, xi_k >= 1 (Kunis &
// Melzer, Section 4, eq. (4.1) with general xi_k), where Algorithm 2's Fourier
// factor A = (exp(2 pi i xi_k x_j)) becomes a transform nonequispaced in both
// time and frequency (an NNFFT, as the proof of Theorem 4.3 notes).
//
// NNFFT of one band (frequencies xi_k <= cut, sorted; centre xc, 2 xc an
// integer; |x| <= 1/2):
//   sum_k u_k exp(2 pi i xi_k x)
//     = exp(2 pi i xc x) sum_k u_k exp(2 pi i (xi_k - xc) x)
//     ~ exp(2 pi i xc x) / Phi(x/2) * sum_g G_g exp(2 pi i g (x/2)),
//   G_g = sum_k u_k phi(g - 2 (xi_k - xc)),
// with phi the Kaiser-Bessel window (half-width m_w, grid spacing 1/2 in
// frequency) and Phi its Fourier transform: by Poisson summation the sampled
// integral of the spread function equals the continuous one up to aliases at
// x/2 + n, n != 0, which the window suppresses exactly as in an NFFT with
// oversampling 2 (|x/2| <= 1/4).  The sum over g is an ordinary NFFT at the
// nodes x/2 (the grid, FFT and gather of the integer path), with its own
// deconvolution 1/Phi(g / n) applied to G_g here.
//
// This file: the plan-time tables (window taps per exponent, the CSR of
// floor(2 xi_k), the 1/Phi tables of the grid sizes) and the frequency
// spreading, written deterministically: one thread per grid frequency sums
// over its exponents in sorted order.
#include <math.h>

#include <algorithm>
#include <vector>

#include "fl_plan.cuh"

namespace fl {

// win[k 2m + t] = phi((bk_k - m + 1 + t) - 2 xi_k), bk_k = floor(2 xi_k), t < 2m.
template <typename T>
__global__ void k_xi_win(int64_t N, const double* __restrict__ xis, int m, double b,
                         int32_t* __restrict__ bk, T* __restrict__ win) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const double x2 = 2.0 * xis[k];
    const double fb = floor(x2);
    bk[k] = (int32_t)fb;
    for (int t = 0; t < 2 * m; ++t)
        win[k * 2 * m + t] = (T)kb_window<double>(fb - m + 1 + t - x2, (double)m, b);
}

// iphi[g] = 1 / Phi(g / n), g = 0 .. count - 1 (count - 1 = the largest occupied
// |g| of the grids of this size, n/4 or a few beyond), Phi(nu) = pi I_0(m sqrt(b^2 - (2 pi nu)^2)).
template <typename T>
__global__ void k_xi_iphi(int64_t count, double n, int m, double b, T* __restrict__ iphi) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    const double nu = 6.283185307179586476925286766559 * (double)g / n;
    iphi[g] = (T)(1.0 / (3.141592653589793238462643383279 * cyl_bessel_i0((double)m * sqrt(fmax(b * b - nu * nu, 0.0)))));
}

// The coefficients in sorted exponent order, once per execute: cs[k] = c[xperm[k]].
template <typename T>
__global__ void k_xi_sortc(int64_t N, const int32_t* __restrict__ xperm, const C_t<T>* __restrict__ c,
                           C_t<T>* __restrict__ cs) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) cs[k] = c[xperm[k]];
}

// QC consecutive weights of one exponent-major row, 16-byte loads (the row
// start is 16-byte aligned: D_off, dld and s0 are multiples of 4).
template <typename T, int QC>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T* d) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int v = 0; v < QC / 4; ++v) {
            const float4 x = __ldg(reinterpret_cast<const float4*>(p) + v);
            d[4 * v] = x.x;
            d[4 * v + 1] = x.y;
            d[4 * v + 2] = x.z;
            d[4 * v + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int v = 0; v < QC / 2; ++v) {
            const double2 x = __ldg(reinterpret_cast<const double2*>(p) + v);
            d[2 * v] = x.x;
            d[2 * v + 1] = x.y;
        }
    }
}

// G of every NNFFT band in one launch: the blocks first_j .. first_{j+1} - 1
// belong to band xsb[j].y (found by binary search over the nsb entries), one
// thread per grid index i of the band, all right-hand sides, written to the
// band grid (zeros outside |g| <= gh):
//   G_s[g] = (1 / Phi(g / n)) sum_k cs_k D[k][s] phi(g - 2 (xi_k - xc)),
// over the sorted exponents whose taps cover g (floor(2 xi_k) in [G - m, G + m),
// G = g + 2 xc, tap t = G + m - 1 - floor(2 xi_k)), in ascending k.  The
// right-hand sides go in chunks of QC: per exponent one window value, one
// coefficient and QC/4 (float) or QC/2 (double) 16-byte weight loads feed
// 2 QC multiply-adds.
template <typename T, int QC>
__global__ void __launch_bounds__(256)
    k_xi_spread(const int2* __restrict__ xsb, int nsb, const BandDev* __restrict__ bands,
                const C_t<T>* __restrict__ cs, const int32_t* __restrict__ xbk,
                const int32_t* __restrict__ xstart, int64_t nstart, const T* __restrict__ win,
                const T* __restrict__ D, const T* __restrict__ iphi, int m, C_t<T>* __restrict__ grid) {
    using C = C_t<T>;
    const int blk = (int)blockIdx.x;
    int lo = 0, hi = nsb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (xsb[mid].x <= blk) lo = mid;
        else hi = mid - 1;
    }
    const int2 sb = xsb[lo];
    const BandDev& B = bands[sb.y];
    const int64_t n = B.n;
    const int64_t i = (int64_t)(blk - sb.x) * 256 + threadIdx.x;
    if (i >= n) return;
    const int nrhs = B.nrhs;
    const int64_t g = i < (n >> 1) ? i : i - n;
    C* out = grid + B.grid_off + i;
    if (g > B.gh || g < -B.gh) {
        for (int s = 0; s < nrhs; ++s) out[(int64_t)s * n] = C{(T)0, (T)0};
        return;
    }
    const int64_t G = g + (int64_t)(2.0 * B.xc);
    const int64_t b0 = std::min<int64_t>(std::max<int64_t>(G - m, 0), nstart - 1);
    const int64_t b1 = std::min<int64_t>(std::max<int64_t>(G + m, 0), nstart - 1);
    const int64_t k0 = xstart[b0];
    const int64_t k1 = std::min<int64_t>(xstart[b1], B.K);
    const T inv = iphi[B.phi_off + (g < 0 ? -g : g)];
    const T* Db = D + B.D_off;
    if (nrhs == 1) {   // one right-hand side, dld = 1
        C acc = {(T)0, (T)0};
        for (int64_t k = k0; k < k1; ++k) {
            const int t = (int)(G + m - 1 - xbk[k]);      // in [0, 2m)
            const T wd = win[k * 2 * m + t] * Db[k];
            const C v = cs[k];
            acc.x += wd * v.x;
            acc.y += wd * v.y;
        }
        out[0] = C{acc.x * inv, acc.y * inv};
        return;
    }
    const int64_t ld = B.dld;   // a multiple of QC
    for (int s0 = 0; s0 < nrhs; s0 += QC) {
        C acc[QC];
#pragma unroll
        for (int u = 0; u < QC; ++u) acc[u] = C{(T)0, (T)0};
        for (int64_t k = k0; k < k1; ++k) {
            const int t = (int)(G + m - 1 - xbk[k]);
            const T wk = win[k * 2 * m + t];
            const C v = cs[k];
            const C wv = C{wk * v.x, wk * v.y};
            T d[QC];
            load_row<T, QC>(Db + k * ld + s0, d);
#pragma unroll
            for (int u = 0; u < QC; ++u) {
                acc[u].x += d[u] * wv.x;
                acc[u].y += d[u] * wv.y;
            }
        }
#pragma unroll
        for (int u = 0; u < QC; ++u)
            if (s0 + u < nrhs) out[(int64_t)(s0 + u) * n] = C{acc[u].x * inv, acc[u].y * inv};
    }
}

// Adjoint of the frequency spreading and of the outer deconvolution, summed
// over the bands (the transpose of k_xi_spread): thread per sorted exponent k,
//   out[xperm[k]] = sum_bands sum_s D[k][s] sum_t phi_t,k / Phi(g_t / n) b_s[g_t mod n],
// g_t = floor(2 xi_k) - m + 1 + t - 2 xc, t < 2m, |g_t| <= gh: exactly the
// (exponent, grid frequency) pairs the forward spreading couples.  The
// exponent's weight row is read in chunks of QC by 16-byte loads, once per
// band and chunk, and kept in registers over the 2m taps.
template <typename T, int QC>
__global__ void __launch_bounds__(256)
    k_xi_combine(int64_t N, int levels, const BandDev* __restrict__ bands,
                 const int32_t* __restrict__ xperm, const int32_t* __restrict__ xbk,
                 const T* __restrict__ win, const T* __restrict__ D, const T* __restrict__ iphi,
                 int m, const C_t<T>* __restrict__ grid, C_t<T>* __restrict__ out) {
    using C = C_t<T>;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int64_t bk = xbk[k];
    const T* wk = win + k * 2 * m;
    C acc = {(T)0, (T)0};
    for (int b = 1; b <= levels; ++b) {
        const BandDev B = bands[b];
        if (B.route != 1 || B.n == 0 || k >= B.K) continue;
        const int64_t c2 = (int64_t)(2.0 * B.xc);
        const T* Dk = D + B.D_off + k * B.dld;
        if (B.nrhs == 1) {   // dld = 1
            const T d = Dk[0];
            for (int t = 0; t < 2 * m; ++t) {
                const int64_t g = bk - m + 1 + t - c2;
                if (g > B.gh || g < -B.gh) continue;
                const T wt = wk[t] * iphi[B.phi_off + (g < 0 ? -g : g)] * d;
                const C v = grid[B.grid_off + (g & (B.n - 1))];
                acc.x += wt * v.x;
                acc.y += wt * v.y;
            }
            continue;
        }
        for (int s0 = 0; s0 < B.nrhs; s0 += QC) {   // dld is a multiple of QC
            T d[QC];
            load_row<T, QC>(Dk + s0, d);
            for (int t = 0; t < 2 * m; ++t) {
                const int64_t g = bk - m + 1 + t - c2;
                if (g > B.gh || g < -B.gh) continue;
                const T wt = wk[t] * iphi[B.phi_off + (g < 0 ? -g : g)];
                const C* gs = grid + B.grid_off + (g & (B.n - 1)) + (int64_t)s0 * B.n;
                C a = {(T)0, (T)0};
#pragma unroll
                for (int u = 0; u < QC; ++u) {
                    if (s0 + u < B.nrhs) {
                        const C v = gs[(int64_t)u * B.n];
                        a.x += d[u] * v.x;
                        a.y += d[u] * v.y;
                    }
                }
                acc.x += wt * a.x;
                acc.y += wt * a.y;
            }
        }
    }
    out[xperm[k]] = acc;
}

template <typename T>
static cudaError_t xi_tables_t(Plan& p, cudaStream_t st) {
    const int64_t N = p.N;
    const int m = p.mw;
    cudaError_t e = cudaMalloc((void**)&p.d_xbk, std::max<int64_t>(N, 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p.d_xwin, std::max<int64_t>(N, 1) * 2 * m * sizeof(T));
    if (e != cudaSuccess) return e;
    if (N > 0)
        k_xi_win<T><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, p.d_xis, m, p.kb_b, p.d_xbk,
                                                                 (T*)p.d_xwin);
    // CSR of floor(2 xi): xstart[B] = first sorted k with floor(2 xi_k) >= B
    const int64_t bmax = N > 0 ? (int64_t)floor(2.0 * p.h_xis.back()) : 0;
    std::vector<int32_t> start(bmax + 2);
    int64_t k = 0;
    for (int64_t B = 0; B <= bmax + 1; ++B) {
        while (k < N && (int64_t)floor(2.0 * p.h_xis[k]) < B) ++k;
        start[B] = (int32_t)k;
    }
    e = cudaMalloc((void**)&p.d_xstart, start.size() * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p.d_xstart, start.data(), start.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    // 1/Phi of every NNFFT grid size (g = 0 .. max(Nm/2, largest gh of the size))
    std::vector<int64_t> off(kMaxLog2n + 1, -1), cnt(kMaxLog2n + 1, 0);
    for (const BandHost& bh : p.bands) {
        const BandDev& d = bh.dev;
        if (d.route != 1 || d.n == 0) continue;
        cnt[d.log2n] = std::max(cnt[d.log2n], std::max(d.Nm / 2, d.gh) + 1);
    }
    int64_t tot = 0;
    for (int lg = 0; lg <= kMaxLog2n; ++lg) {
        if (cnt[lg] == 0) continue;
        off[lg] = tot;
        tot += cnt[lg];
    }
    for (BandHost& bh : p.bands) {
        BandDev& d = bh.dev;
        if (d.route != 1 || d.n == 0) continue;
        d.phi_off = off[d.log2n];
    }
    p.xiphi_elems = tot;
    if (tot > 0) {
        e = cudaMalloc(&p.d_xiphi, tot * sizeof(T));
        if (e != cudaSuccess) return e;
        for (int lg = 0; lg <= kMaxLog2n; ++lg) {
            if (off[lg] < 0) continue;
            const int64_t n = (int64_t)1 << lg;
            k_xi_iphi<T><<<(unsigned)((cnt[lg] + 255) / 256), 256, 0, st>>>(cnt[lg], (double)n, m, p.kb_b,
                                                                            (T*)p.d_xiphi + off[lg]);
        }
    }
    // the spreading launch: its NNFFT bands in order with their first blocks
    std::vector<int2> sb;
    int64_t blocks = 0;
    for (size_t b = 0; b < p.bands.size(); ++b) {
        const BandDev& d = p.bands[b].dev;
        if (d.route != 1 || d.n == 0) continue;
        sb.push_back(make_int2((int)blocks, (int)b));
        blocks += (d.n + 255) / 256;
    }
    if (blocks > INT32_MAX) return cudaErrorInvalidValue;
    p.xsb_n = (int)sb.size();
    p.xsb_blocks = blocks;
    if (!sb.empty()) {
        e = cudaMalloc((void**)&p.d_xsb, sb.size() * sizeof(int2));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p.d_xsb, sb.data(), sb.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    e = cudaMalloc(&p.d_xcs, std::max<int64_t>(N, 1) * sizeof(C_t<T>));
    if (e != cudaSuccess) return e;
    // the band table with phi_off
    std::vector<BandDev> hb(p.bands.size());
    for (size_t b = 0; b < p.bands.size(); ++b) hb[b] = p.bands[b].dev;
    e = cudaMemcpyAsync(p.d_bands, hb.data(), hb.size() * sizeof(BandDev), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t build_xi_tables(Plan& p, cudaStream_t st) {
    return p.prec == FL_FP64 ? xi_tables_t<double>(p, st) : xi_tables_t<float>(p, st);
}

template <typename T, int QC>
static void xi_spread_launch(Plan& p, int64_t nstart, cudaStream_t st) {
    k_xi_spread<T, QC><<<(unsigned)p.xsb_blocks, 256, 0, st>>>(
        p.d_xsb, p.xsb_n, p.d_bands, (const C_t<T>*)p.d_xcs, p.d_xbk, p.d_xstart, nstart,
        (const T*)p.d_xwin, (const T*)p.d_D, (const T*)p.d_xiphi, p.mw, (C_t<T>*)p.d_grid);
}

template <typename T>
static cudaError_t xi_spread_t(Plan& p, const void* c, cudaStream_t st) {
    using C = C_t<T>;
    const int64_t nstart = p.N > 0 ? (int64_t)floor(2.0 * p.h_xis.back()) + 2 : 1;
    // algorithmic bytes: the sorted coefficients (gather + write + read), each
    // exponent's taps and weight row once per band, the grids written
    double bytes = (double)p.N * (3 * sizeof(C) + 4);
    for (const BandHost& bh : p.bands) {
        const BandDev& d = bh.dev;
        if (d.route != 1 || d.n == 0) continue;
        bytes += (double)d.K * (4 + 2 * p.mw * sizeof(T) + d.dld * sizeof(T)) +
                 (double)d.nrhs * d.n * sizeof(C);
    }
    int slot;
    timer_begin(p, "xi_spread", bytes, st, &slot);
    if (p.N > 0) {
        k_xi_sortc<T><<<(unsigned)((p.N + 255) / 256), 256, 0, st>>>(p.N, p.d_xperm, (const C*)c,
                                                                      (C*)p.d_xcs);
        ++p.launches;
    }
    if (p.xsb_blocks > 0) {
        switch (p.xqc) {
        case 4: xi_spread_launch<T, 4>(p, nstart, st); break;
        case 8: xi_spread_launch<T, 8>(p, nstart, st); break;
        case 12: xi_spread_launch<T, 12>(p, nstart, st); break;
        default: xi_spread_launch<T, 16>(p, nstart, st); break;
        }
        ++p.launches;
    }
    timer_end(p, slot, st);
    return cudaGetLastError();
}

cudaError_t launch_xi_spread(Plan& p, const void* c, cudaStream_t st) {
    return p.prec == FL_FP64 ? xi_spread_t<double>(p, c, st) : xi_spread_t<float>(p, c, st);
}

template <typename T, int QC>
static void xi_combine_launch(Plan& p, void* out, cudaStream_t st) {
    k_xi_combine<T, QC><<<(unsigned)((p.N + 255) / 256), 256, 0, st>>>(
        p.N, p.levels, p.d_bands, p.d_xperm, p.d_xbk, (const T*)p.d_xwin, (const T*)p.d_D,
        (const T*)p.d_xiphi, p.mw, (const C_t<T>*)p.d_grid, (C_t<T>*)out);
}

template <typename T>
static cudaError_t xi_combine_t(Plan& p, void* out, cudaStream_t st) {
    int slot;
    timer_begin(p, "combine", 0.0, st, &slot);
    switch (p.xqc) {
    case 4: xi_combine_launch<T, 4>(p, out, st); break;
    case 8: xi_combine_launch<T, 8>(p, out, st); break;
    case 12: xi_combine_launch<T, 12>(p, out, st); break;
    default: xi_combine_launch<T, 16>(p, out, st); break;
    }
    timer_end(p, slot, st);
    ++p.launches;
    return cudaGetLastError();
}

cudaError_t launch_xi_combine(Plan& p, void* out, cudaStream_t st) {
    return p.prec == FL_FP64 ? xi_combine_t<double>(p, out, st) : xi_combine_t<float>(p, out, st);
}

}  // namespace fl
