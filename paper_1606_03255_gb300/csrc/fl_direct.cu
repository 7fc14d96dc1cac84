// fl_direct.cu -- direct evaluation of the bands whose node count is too small
// to pay for an NFFT with q right-hand sides, and of their adjoint.
//
// A band routed here computes the plain sum f_j = sum_{k<K} c_k z_j^k over the
// frequencies the band keeps (K = k <= xi_1 / 2^(l_m - 1), the region-(ii)
// truncation of Lemma A.2, or K = N for the Y_M band), i.e. eq. (4.1) itself
// -- the "naive matrix vector multiplication" the paper times in Section 5 --
// restricted to those frequencies.  The sum is blocked: each block of 32 terms
// is a Horner polynomial in z_j, and z_j^{k_b} at the block start is formed
// from an exactly reduced phase (k_b x_j mod 1) and exp(-y_j k_b), so the error
// does not grow with k.
#include "fl_ffmath.cuh"
#include "fl_plan.cuh"

namespace fl {

constexpr double kTwoPiDir = 6.283185307179586476925286766559;

// Shared-memory stride of a staged Horner block: one element of padding, so
// the 32 lanes of a warp, each on its own block, read 32 different bank
// offsets instead of one (blocks of 32 complex values are 256 or 512 bytes
// apart, a whole number of bank rows).
constexpr int kDirBlockLd = kDirBlock + 1;
constexpr int kDirTile = kDirChunk / kDirBlock * kDirBlockLd;

// frac(k x) in [-1/2, 1/2) for the FP64 form and the float pairs: k x = p + e
// exactly (FMA), one rounding.  (The FP32 form uses dir_f32_power below.)
template <typename T> __device__ __forceinline__ double dir_phase(double k, double x);
template <> __device__ __forceinline__ double dir_phase<double>(double k, double x) {
    return frac_turns(k, x);
}

template <typename T> __device__ __forceinline__ T dir_exp(T a);
template <> __device__ __forceinline__ float dir_exp<float>(float a) { return expf(a); }
template <> __device__ __forceinline__ double dir_exp<double>(double a) { return exp(a); }

// FP32 form without FP64 arithmetic per block: x in [0, 1) held as the 64-bit
// fixed-point X = x 2^64 (exact for the 53-bit x), so frac(k x) is the
// wrapped product k X, rounded to 24 bits and read as a signed value in
// [-1/2, 1/2); y as a float pair (hi + lo), so y k = p + e with p = fl(hi k)
// and e its error plus lo k, and exp(-y k) = exp(-p) (1 - e) (|e| < 2^-20 p).
struct DirF32Node {
    uint64_t X;
    float yh, yl;
};

// A node from the plan's record (k_node_tab: X = x 2^64, and y = 2 pi Im w as
// a float pair, formed once at plan time in double), with z = exp(-y)
// e^(2 pi i x) in float: x - [x >= 1/2] is the signed X 2^-64, rounded once
// to float.
__device__ __forceinline__ DirF32Node dir_f32_record(uint4 rec, float2* z) {
    DirF32Node d;
    d.X = ((uint64_t)rec.y << 32) | (uint64_t)rec.x;
    d.yh = __uint_as_float(rec.z);
    d.yl = __uint_as_float(rec.w);
    const float xr = (float)(int64_t)d.X * 0x1p-64f;
    *z = cscale(expipi<float>(2.f * xr), expf(-d.yh));
    return d;
}

// z^k = exp(-y k) e^(2 pi i frac(k x)) for 0 <= k < 2^24 (SIGN = -1: the conjugate
// phase); false when y k > lim (the power underflows: so do all later ones).
template <int SIGN>
__device__ __forceinline__ bool dir_f32_power(const DirF32Node& d, int64_t k, float lim, float2* zk) {
    const float kf = (float)k;                 // exact: k < 2^24
    const float p = d.yh * kf;
    if (p > lim) return false;
    const float e = fmaf(d.yh, kf, -p) + d.yl * kf;
    const float mag = expf(-p) * (1.f - e);
    const uint64_t ph = (uint64_t)k * d.X + (1ull << 39);
    const float phase = (float)((int64_t)ph >> 40) * 0x1p-24f;   // frac(k x) in [-1/2, 1/2)
    *zk = cscale(expipi<float>((float)(2 * SIGN) * phase), mag);
    return true;
}

// Warp part of k_direct for node w of the item: lane l sums the Horner blocks
// l, l + 32, ... of the staged chunk; lane 0 writes the node's partial.
template <typename T>
__device__ __forceinline__ void direct_node(const DirectItem& it, const BandDev& B, const C_t<T>* tile,
                                            const double2* __restrict__ ws,
                                            const uint4* __restrict__ ntab, int64_t k0, int64_t kend,
                                            int w, int lane, C_t<T>* __restrict__ part) {
    using C = C_t<T>;
    const int64_t i = it.node0 + w;
    // z = exp(-y) exp(2 pi i x) in T (FP32: from the node record)
    C z;
    DirF32Node nd;
    double x = 0.0, y = 0.0;
    if constexpr (sizeof(T) == 4) {
        nd = dir_f32_record(ntab[i], &z);
    } else {
        const double2 wv = ws[i];
        x = wv.x - floor(wv.x);
        y = kTwoPiDir * wv.y;
        const double xr = x >= 0.5 ? x - 1.0 : x;
        z = cscale(expipi<T>((T)(2.0 * xr)), dir_exp<T>((T)(-y)));
    }
    C acc = C{(T)0, (T)0};
#pragma unroll 1
    for (int bb = 0; bb < kDirChunk / (32 * kDirBlock); ++bb) {
        const int b = bb * 32 + lane;
        const int64_t kb = k0 + (int64_t)b * kDirBlock;
        if (kb >= kend) break;
        C zk;
        if constexpr (sizeof(T) == 4) {
            if (!dir_f32_power<1>(nd, kb, 104.f, &zk)) break;   // z^kb underflows: so do later blocks
        } else {
            const double ykb = y * (double)kb;
            if (ykb > 745.0) break;
            zk = cscale(expipi<T>((T)(2.0 * dir_phase<T>((double)kb, x))), dir_exp<T>((T)(-ykb)));
        }
        const C* cb = tile + b * kDirBlockLd;
        C P = cb[kDirBlock - 1];
#pragma unroll
        for (int t = kDirBlock - 2; t >= 0; --t) P = cadd(cmul(P, z), cb[t]);
        acc = cadd(acc, cmul(zk, P));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) part[B.dslot + (i - B.node_off) * B.nchunk + it.chunk] = acc;
}

// One CTA per work item: up to kDirNodes consecutive sorted nodes of one band
// against one chunk of kDirChunk coefficients staged in shared memory.  Warp w
// takes nodes w, w + 8, ...; lane l the Horner blocks l, l + 32, ... of the
// chunk.
template <typename T, bool DERIV>
__global__ void __launch_bounds__(256) k_direct(const DirectItem* __restrict__ items,
                                                const BandDev* __restrict__ bands,
                                                const double2* __restrict__ ws,
                                                const uint4* __restrict__ ntab,
                                                const C_t<T>* __restrict__ c,
                                                C_t<T>* __restrict__ part) {
    using C = C_t<T>;
    extern __shared__ unsigned char smem_raw[];
    C* tile = reinterpret_cast<C*>(smem_raw);
    const DirectItem it = items[blockIdx.x];
    const BandDev B = bands[it.band];
    const int64_t k0 = (int64_t)it.chunk * kDirChunk;
    const int64_t kend = min(B.K, k0 + (int64_t)kDirChunk);
    // the chunk's terms rounded up to whole Horner blocks (zeros past kend)
    const int nst = (int)((kend - k0 + kDirBlock - 1) / kDirBlock) * kDirBlock;
    for (int i = threadIdx.x; i < nst; i += blockDim.x) {
        const int64_t k = k0 + i;
        C v = C{(T)0, (T)0};
        if (k < kend) {
            v = c[B.c_off + k];
            if (DERIV) {
                T wgt;
                if constexpr (sizeof(T) == 4) wgt = (float)k * 6.28318530717958647692f;   // k < 2^24: one rounding
                else wgt = kTwoPiDir * (double)k;
                v = C{-v.y * wgt, v.x * wgt};
            }
        }
        tile[i + i / kDirBlock] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int w = threadIdx.x >> 5; w < it.nnodes; w += 8)
        direct_node<T>(it, B, tile, ws, ntab, k0, kend, w, lane, part);
}

// Bands with K <= kDirSmallK: one thread per node (up to kDirSmallNodes per
// CTA), the band's K coefficients staged once, all K terms per thread in the
// same blocked Horner form (blocks of kDirBlock terms from an exactly reduced
// power z^kb); the partial of chunk 0 as for k_direct.
template <typename T, bool DERIV>
__global__ void __launch_bounds__(kDirSmallNodes) k_direct_small(const DirectItem* __restrict__ items,
                                                                 const BandDev* __restrict__ bands,
                                                                 const double2* __restrict__ ws,
                                                                 const uint4* __restrict__ ntab,
                                                                 const C_t<T>* __restrict__ c,
                                                                 C_t<T>* __restrict__ part) {
    using C = C_t<T>;
    __shared__ C tile[kDirSmallK];
    const DirectItem it = items[blockIdx.x];
    const BandDev B = bands[it.band];
    const int K = (int)B.K;                              // <= kDirSmallK
    const int Kr = (K + kDirBlock - 1) / kDirBlock * kDirBlock;
    for (int k = threadIdx.x; k < Kr; k += blockDim.x) {
        C v = C{(T)0, (T)0};
        if (k < K) {
            v = c[B.c_off + k];
            if (DERIV) {
                T wgt;
                if constexpr (sizeof(T) == 4) wgt = (float)k * 6.28318530717958647692f;
                else wgt = kTwoPiDir * (double)k;
                v = C{-v.y * wgt, v.x * wgt};
            }
        }
        tile[k] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x >= it.nnodes) return;
    const int64_t i = it.node0 + threadIdx.x;
    C z;
    DirF32Node nd;
    double x = 0.0, y = 0.0;
    if constexpr (sizeof(T) == 4) {
        nd = dir_f32_record(ntab[i], &z);
    } else {
        const double2 wv = ws[i];
        x = wv.x - floor(wv.x);
        y = kTwoPiDir * wv.y;
        const double xr = x >= 0.5 ? x - 1.0 : x;
        z = cscale(expipi<T>((T)(2.0 * xr)), dir_exp<T>((T)(-y)));
    }
    C acc = C{(T)0, (T)0};
    for (int kb = 0; kb < K; kb += kDirBlock) {
        C zk;
        if constexpr (sizeof(T) == 4) {
            if (!dir_f32_power<1>(nd, kb, 104.f, &zk)) break;
        } else {
            const double ykb = y * (double)kb;
            if (ykb > 745.0) break;
            zk = cscale(expipi<T>((T)(2.0 * dir_phase<T>((double)kb, x))), dir_exp<T>((T)(-ykb)));
        }
        const C* cb = tile + kb;
        C P = cb[kDirBlock - 1];
#pragma unroll
        for (int t = kDirBlock - 2; t >= 0; --t) P = cadd(cmul(P, z), cb[t]);
        acc = cadd(acc, cmul(zk, P));
    }
    part[B.dslot + (i - B.node_off) * B.nchunk] = acc;
}

// The direct band holding flattened node t: the last range whose prefix is
// <= t (prefixes ascend; binary search, so batches of thousands of direct
// bands cost log2 of that per node).
__device__ __forceinline__ int find_direct_range(const DirectRange* __restrict__ ranges, int nranges,
                                                 int64_t t) {
    int lo = 0, hi = nranges;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ranges[mid].prefix <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// f[perm[i]] = sum over the node's chunks (in chunk order); with rmul,
// rmul[perm[i]] * conj(sum) (the node-gradient epilogue).
template <typename T>
__global__ void k_direct_reduce(int nranges, const DirectRange* __restrict__ ranges,
                                int64_t total, const BandDev* __restrict__ bands,
                                const int32_t* __restrict__ perm, const C_t<T>* __restrict__ part,
                                const C_t<T>* __restrict__ rmul, C_t<T>* __restrict__ f) {
    using C = C_t<T>;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const DirectRange R = ranges[find_direct_range(ranges, nranges, t)];
    const BandDev B = bands[R.band];
    const int64_t local = t - R.prefix;
    const C* p = part + B.dslot + local * B.nchunk;
    C acc = C{(T)0, (T)0};
    for (int ch = 0; ch < B.nchunk; ++ch) acc = cadd(acc, p[ch]);
    const int32_t j = perm[B.node_off + local];
    f[j] = rmul ? cmulc(rmul[j], acc) : acc;
}

// Adjoint of the direct bands, cdir[k] += sum_{j in band} r_j conj(z_j)^k for
// k < K_b: the transpose of the blocked Horner sum.  One warp per work item
// (band, chunk of 32 KL frequencies, up to kDirAdjNodes nodes); lane l owns
// the KL frequencies k0 = chunk 32 KL + l KL .. k0 + KL - 1.  For each node
// (broadcast across the warp by shuffles) the lane forms conj(z_j)^k0 from an
// exactly reduced phase, then steps through its frequencies multiplying by
// conj(z_j).  Chunks of different node groups meet in cdir through atomics.
template <typename T> struct AdjKL { static constexpr int KL = sizeof(T) == 4 ? 32 : 16; };

template <typename T>
__global__ void __launch_bounds__(32) k_direct_adj(const DirectAdjItem* __restrict__ items,
                                                   const BandDev* __restrict__ bands,
                                                   const double2* __restrict__ ws,
                                                   const uint4* __restrict__ ntab,
                                                   const int32_t* __restrict__ perm,
                                                   const C_t<T>* __restrict__ r,
                                                   C_t<T>* __restrict__ cdir) {
    using C = C_t<T>;
    constexpr int KL = AdjKL<T>::KL;
    const DirectAdjItem it = items[blockIdx.x];
    const BandDev B = bands[it.band];
    const int lane = threadIdx.x;
    const int64_t k0 = (int64_t)it.kchunk * (32 * KL) + (int64_t)lane * KL;
    const bool active = k0 < B.K;
    C acc[KL];
#pragma unroll
    for (int t = 0; t < KL; ++t) acc[t] = C{(T)0, (T)0};
    for (int nb = 0; nb < it.nnodes; nb += 32) {
        // lane loads node nb + lane: x, y, r_j and conj(z_j) in T
        double xl = 0.0, yl = 0.0;
        C rl = C{(T)0, (T)0}, zl = C{(T)0, (T)0};
        DirF32Node nl = {0ull, 0.f, 0.f};
        if (nb + lane < it.nnodes) {
            const int64_t i = it.node0 + nb + lane;
            rl = r[perm[i]];
            if constexpr (sizeof(T) == 4) {   // from the node record; conj(z)
                nl = dir_f32_record(ntab[i], &zl);
                zl.y = -zl.y;
            } else {
                const double2 wv = ws[i];
                xl = wv.x - floor(wv.x);
                yl = kTwoPiDir * wv.y;
                const double xr = xl >= 0.5 ? xl - 1.0 : xl;
                zl = cscale(expipi<T>((T)(-2.0 * xr)), dir_exp<T>((T)(-yl)));
            }
        }
        const int cnt = min(32, it.nnodes - nb);
        for (int q = 0; q < cnt; ++q) {
            const C rq = C{__shfl_sync(0xffffffffu, rl.x, q), __shfl_sync(0xffffffffu, rl.y, q)};
            const C zq = C{__shfl_sync(0xffffffffu, zl.x, q), __shfl_sync(0xffffffffu, zl.y, q)};
            C w0;
            if constexpr (sizeof(T) == 4) {
                DirF32Node nq;
                nq.X = ((uint64_t)__shfl_sync(0xffffffffu, (unsigned)(nl.X >> 32), q) << 32) |
                       (uint64_t)__shfl_sync(0xffffffffu, (unsigned)nl.X, q);
                nq.yh = __shfl_sync(0xffffffffu, nl.yh, q);
                nq.yl = __shfl_sync(0xffffffffu, nl.yl, q);
                if (!active) continue;
                if (!dir_f32_power<-1>(nq, k0, 104.f, &w0)) continue;
            } else {
                const double x = __shfl_sync(0xffffffffu, xl, q);
                const double y = __shfl_sync(0xffffffffu, yl, q);
                if (!active) continue;
                const double yk = y * (double)k0;
                if (yk > 745.0) continue;
                w0 = cscale(expipi<T>((T)(-2.0 * dir_phase<T>((double)k0, x))), dir_exp<T>((T)(-yk)));
            }
            C rw = cmul(rq, w0);
#pragma unroll
            for (int t = 0; t < KL; ++t) {
                acc[t] = cadd(acc[t], rw);
                rw = cmul(rw, zq);
            }
        }
    }
    if (!active) return;
#pragma unroll
    for (int t = 0; t < KL; ++t) {
        const int64_t k = k0 + t;
        if (k < B.K) {
            atomicAdd(&cdir[k].x, acc[t].x);
            atomicAdd(&cdir[k].y, acc[t].y);
        }
    }
}

// The float-pair form (FL_FP64_FF): k_direct with the Horner steps, the
// block-start powers z_j^kb = exp(-y kb) e^(2 pi i frac(kb x)) and the sums in
// float pairs (fl_ffmath.cuh); the phases kb x are still reduced exactly in
// double.  c: the coefficients already converted to pairs.
__global__ void __launch_bounds__(256) k_direct_ff(const DirectItem* __restrict__ items,
                                                   const BandDev* __restrict__ bands,
                                                   const double2* __restrict__ ws,
                                                   const ffc* __restrict__ c,
                                                   ffc* __restrict__ part) {
    extern __shared__ unsigned char smem_raw[];
    ffc* tile = reinterpret_cast<ffc*>(smem_raw);
    const DirectItem it = items[blockIdx.x];
    const BandDev B = bands[it.band];
    const int64_t k0 = (int64_t)it.chunk * kDirChunk;
    const int64_t kend = min(B.K, k0 + (int64_t)kDirChunk);
    const int nst = (int)((kend - k0 + kDirBlock - 1) / kDirBlock) * kDirBlock;
    for (int i = threadIdx.x; i < nst; i += blockDim.x) {
        const int64_t k = k0 + i;
        tile[i + i / kDirBlock] = k < kend ? c[B.c_off + k] : ffc{ff(0), ff(0)};
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int w = threadIdx.x >> 5; w < it.nnodes; w += 8) {   // nodes w, w + 8, ...
        const int64_t i = it.node0 + w;
        const double2 wv = ws[i];
        const double x = wv.x - floor(wv.x);
        const double y = kTwoPiDir * wv.y;
        double xr = x;
        if (xr >= 0.5) xr -= 1.0;
        ffc z;
        ff_sincospi(ff(2.0 * xr), &z.y, &z.x);
        const ff mag = ff_exp(ff(-y));
        z = ffc{z.x * mag, z.y * mag};
        ffc acc = {ff(0), ff(0)};
#pragma unroll 1
        for (int bb = 0; bb < kDirChunk / (32 * kDirBlock); ++bb) {
            const int b = bb * 32 + lane;
            const int64_t kb = k0 + (int64_t)b * kDirBlock;
            if (kb >= kend) break;
            const double ykb = y * (double)kb;
            if (ykb > 104.0) break;     // below 2^-150 |c|: so are the later blocks
            const ffc* cb = tile + b * kDirBlockLd;
            ffc P = cb[kDirBlock - 1];
#pragma unroll
            for (int t = kDirBlock - 2; t >= 0; --t) P = cadd(cmul(P, z), cb[t]);
            ffc zk;
            ff_sincospi(ff(2.0 * dir_phase<double>((double)kb, x)), &zk.y, &zk.x);
            const ff mk = ff_exp(ff(-ykb));
            acc = cadd(acc, cmul(ffc{zk.x * mk, zk.y * mk}, P));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const ffc o = {ff(__shfl_xor_sync(0xffffffffu, acc.x.hi, off),
                              __shfl_xor_sync(0xffffffffu, acc.x.lo, off)),
                           ff(__shfl_xor_sync(0xffffffffu, acc.y.hi, off),
                              __shfl_xor_sync(0xffffffffu, acc.y.lo, off))};
            acc = cadd(acc, o);
        }
        if (lane == 0) part[B.dslot + (i - B.node_off) * B.nchunk + it.chunk] = acc;
    }
}

// f[perm[i]] = sum over the node's chunks (in chunk order), rounded to double.
__global__ void k_direct_reduce_ff(int nranges, const DirectRange* __restrict__ ranges,
                                   int64_t total, const BandDev* __restrict__ bands,
                                   const int32_t* __restrict__ perm, const ffc* __restrict__ part,
                                   const double2* __restrict__ rmul, double2* __restrict__ f) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const DirectRange R = ranges[find_direct_range(ranges, nranges, t)];
    const BandDev B = bands[R.band];
    const int64_t local = t - R.prefix;
    const ffc* p = part + B.dslot + local * B.nchunk;
    ffc acc = {ff(0), ff(0)};
    for (int ch = 0; ch < B.nchunk; ++ch) acc = cadd(acc, p[ch]);
    const int32_t j = perm[B.node_off + local];
    const double2 v = double2{(double)acc.x, (double)acc.y};
    // with rmul: rmul[j] conj(v) (node gradient)
    f[j] = rmul ? cmulc(rmul[j], v) : v;
}

// (the coefficients are read as pairs from p.d_cff, k-weighted by the caller
// for the derivative)
static cudaError_t direct_forward_ff(Plan& p, void* f, const void* rmul, cudaStream_t st) {
    if (p.direct_work.empty()) return cudaSuccess;
    const size_t smem = (size_t)kDirTile * sizeof(ffc);
    cudaError_t e = cudaFuncSetAttribute(k_direct_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int slot;
    timer_begin(p, "direct", (double)p.direct_terms * sizeof(ffc) / 32.0, st, &slot);
    k_direct_ff<<<(unsigned)p.direct_work.size(), 256, smem, st>>>(p.d_direct, p.d_bands, p.d_ws,
                                                                  (const ffc*)p.d_cff, (ffc*)p.d_dpart);
    k_direct_reduce_ff<<<(unsigned)((p.direct_nodes + 255) / 256), 256, 0, st>>>(
        (int)p.direct_ranges.size(), p.d_dranges, p.direct_nodes, p.d_bands, p.d_perm,
        (const ffc*)p.d_dpart, (const double2*)rmul, (double2*)f);
    timer_end(p, slot, st);
    p.launches += 2;
    return cudaGetLastError();
}

// Adjoint of the bands with K <= kDirSmallK: one warp per (band, group of up
// to kDirAdjNodes nodes).  The lanes split into KB blocks of KL frequencies
// (KB the smallest power of two with KB KL >= K) and G = 32 / KB node
// subgroups; each lane sums its subgroup's nodes (every G-th) over its KL
// frequencies, a fixed shuffle tree adds the subgroups, and the first
// subgroup adds the result to cdir (atomics across node groups, as k_direct_adj).
template <typename T>
__global__ void __launch_bounds__(32) k_direct_adj_small(const DirectAdjItem* __restrict__ items,
                                                         const BandDev* __restrict__ bands,
                                                         const double2* __restrict__ ws,
                                                         const uint4* __restrict__ ntab,
                                                         const int32_t* __restrict__ perm,
                                                         const C_t<T>* __restrict__ r,
                                                         C_t<T>* __restrict__ cdir) {
    using C = C_t<T>;
    constexpr int KL = AdjKL<T>::KL;
    const DirectAdjItem it = items[blockIdx.x];
    const BandDev B = bands[it.band];
    const int K = (int)B.K;
    int lkb = 0;
    while ((KL << lkb) < K) ++lkb;                 // KB = 2^lkb <= 32 (K <= kDirSmallK)
    const int lane = threadIdx.x, g = lane >> lkb, G = 32 >> lkb;
    const int64_t k0 = (int64_t)(lane & ((1 << lkb) - 1)) * KL;
    const bool active = k0 < K;
    C acc[KL];
#pragma unroll
    for (int t = 0; t < KL; ++t) acc[t] = C{(T)0, (T)0};
    for (int jn = g; active && jn < it.nnodes; jn += G) {
        const int64_t i = it.node0 + jn;
        C zq, w0;
        double x = 0.0, y = 0.0;
        if constexpr (sizeof(T) == 4) {   // from the node record; conj(z)
            const DirF32Node nd = dir_f32_record(ntab[i], &zq);
            zq.y = -zq.y;
            if (!dir_f32_power<-1>(nd, k0, 104.f, &w0)) continue;
        } else {
            const double2 wv = ws[i];
            x = wv.x - floor(wv.x);
            y = kTwoPiDir * wv.y;
            const double xr = x >= 0.5 ? x - 1.0 : x;
            zq = cscale(expipi<T>((T)(-2.0 * xr)), dir_exp<T>((T)(-y)));
            const double yk = y * (double)k0;
            if (yk > 745.0) continue;
            w0 = cscale(expipi<T>((T)(-2.0 * dir_phase<T>((double)k0, x))), dir_exp<T>((T)(-yk)));
        }
        C rw = cmul(r[perm[i]], w0);
#pragma unroll
        for (int t = 0; t < KL; ++t) {
            acc[t] = cadd(acc[t], rw);
            rw = cmul(rw, zq);
        }
    }
    for (int off = 1 << lkb; off < 32; off <<= 1) {
#pragma unroll
        for (int t = 0; t < KL; ++t) {
            acc[t].x += __shfl_xor_sync(0xffffffffu, acc[t].x, off);
            acc[t].y += __shfl_xor_sync(0xffffffffu, acc[t].y, off);
        }
    }
    if (g != 0 || !active) return;
#pragma unroll
    for (int t = 0; t < KL; ++t) {
        const int64_t k = k0 + t;
        if (k < K) {
            atomicAdd(&cdir[k].x, acc[t].x);
            atomicAdd(&cdir[k].y, acc[t].y);
        }
    }
}

template <typename T>
static cudaError_t direct_forward_t(Plan& p, const void* c, void* f, bool deriv, const void* rmul,
                                    cudaStream_t st) {
    using C = C_t<T>;
    if (p.direct_work.empty()) return cudaSuccess;
    const size_t smem = (size_t)kDirTile * sizeof(C);
    auto kern = deriv ? k_direct<T, true> : k_direct<T, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int slot;
    timer_begin(p, "direct", (double)p.direct_terms * sizeof(C) / 32.0, st, &slot);
    const int64_t nbig = (int64_t)p.direct_work.size() - p.n_direct_small;
    if (nbig > 0)
        kern<<<(unsigned)nbig, 256, smem, st>>>(p.d_direct, p.d_bands, p.d_ws, p.d_ntab, (const C*)c,
                                                (C*)p.d_dpart);
    if (p.n_direct_small > 0) {
        auto ks = deriv ? k_direct_small<T, true> : k_direct_small<T, false>;
        ks<<<(unsigned)p.n_direct_small, kDirSmallNodes, 0, st>>>(p.d_direct + nbig, p.d_bands, p.d_ws,
                                                                  p.d_ntab, (const C*)c, (C*)p.d_dpart);
        ++p.launches;
    }
    k_direct_reduce<T><<<(unsigned)((p.direct_nodes + 255) / 256), 256, 0, st>>>(
        (int)p.direct_ranges.size(), p.d_dranges, p.direct_nodes, p.d_bands, p.d_perm,
        (const C*)p.d_dpart, (const C*)rmul, (C*)f);
    timer_end(p, slot, st);
    p.launches += 1 + (nbig > 0);
    return cudaGetLastError();
}

cudaError_t run_direct_forward(Plan& p, const void* c, void* f, bool deriv, const void* rmul,
                               cudaStream_t st) {
    if (p.prec == FL_FP64_FF)   // reads the coefficients as pairs (converted by the caller)
        return direct_forward_ff(p, f, rmul, st);
    return p.prec == FL_FP64 ? direct_forward_t<double>(p, c, f, deriv, rmul, st)
                             : direct_forward_t<float>(p, c, f, deriv, rmul, st);
}

// The float-pair form's adjoint of the direct bands with K > kDirSmallK:
// k_direct_adj's steps (same work items, KL = 16 frequencies per lane) with
// conj(z_j), the restart power conj(z_j)^k0 and the frequency steps in float
// pairs; the restart phase k0 x mod 1 is still reduced exactly in double.
// Each lane's sums, rounded to double, meet in cdir through atomics.
__global__ void __launch_bounds__(32) k_direct_adj_ff(const DirectAdjItem* __restrict__ items,
                                                      const BandDev* __restrict__ bands,
                                                      const double2* __restrict__ ws,
                                                      const int32_t* __restrict__ perm,
                                                      const double2* __restrict__ r,
                                                      double2* __restrict__ cdir) {
    constexpr int KL = 16;
    const DirectAdjItem it = items[blockIdx.x];
    const BandDev B = bands[it.band];
    const int lane = threadIdx.x;
    const int64_t k0 = (int64_t)it.kchunk * (32 * KL) + (int64_t)lane * KL;
    const bool active = k0 < B.K;
    ffc acc[KL];
#pragma unroll
    for (int t = 0; t < KL; ++t) acc[t] = ffc{ff(0), ff(0)};
    for (int nb = 0; nb < it.nnodes; nb += 32) {
        // lane loads node nb + lane: x, y, r_j and conj(z_j) as pairs
        double xl = 0.0, yl = 0.0;
        ffc rl = {ff(0), ff(0)}, zl = {ff(0), ff(0)};
        if (nb + lane < it.nnodes) {
            const int64_t i = it.node0 + nb + lane;
            const double2 wv = ws[i];
            xl = wv.x - floor(wv.x);
            yl = kTwoPiDir * wv.y;
            const double2 rv = r[perm[i]];
            rl = ffc{ff(rv.x), ff(rv.y)};
            const double xr = xl >= 0.5 ? xl - 1.0 : xl;
            ff_sincospi(ff(-2.0 * xr), &zl.y, &zl.x);
            const ff mag = ff_exp(ff(-yl));
            zl = ffc{zl.x * mag, zl.y * mag};
        }
        const int cnt = min(32, it.nnodes - nb);
        for (int q = 0; q < cnt; ++q) {
            const ffc rq = {ff(__shfl_sync(0xffffffffu, rl.x.hi, q), __shfl_sync(0xffffffffu, rl.x.lo, q)),
                            ff(__shfl_sync(0xffffffffu, rl.y.hi, q), __shfl_sync(0xffffffffu, rl.y.lo, q))};
            const ffc zq = {ff(__shfl_sync(0xffffffffu, zl.x.hi, q), __shfl_sync(0xffffffffu, zl.x.lo, q)),
                            ff(__shfl_sync(0xffffffffu, zl.y.hi, q), __shfl_sync(0xffffffffu, zl.y.lo, q))};
            const double x = __shfl_sync(0xffffffffu, xl, q);
            const double y = __shfl_sync(0xffffffffu, yl, q);
            if (!active) continue;
            const double yk = y * (double)k0;
            if (yk > 104.0) continue;   // below 2^-150 |r_j|
            ffc w0;
            ff_sincospi(ff(-2.0 * dir_phase<double>((double)k0, x)), &w0.y, &w0.x);
            const ff mk = ff_exp(ff(-yk));
            ffc rw = cmul(rq, ffc{w0.x * mk, w0.y * mk});
#pragma unroll
            for (int t = 0; t < KL; ++t) {
                acc[t] = cadd(acc[t], rw);
                rw = cmul(rw, zq);
            }
        }
    }
    if (!active) return;
#pragma unroll
    for (int t = 0; t < KL; ++t) {
        const int64_t k = k0 + t;
        if (k < B.K) {
            atomicAdd(&cdir[k].x, (double)acc[t].x);
            atomicAdd(&cdir[k].y, (double)acc[t].y);
        }
    }
}

// (pairs: the float-pair form, T = double, whose bands with K > kDirSmallK
// take k_direct_adj_ff)
template <typename T>
static cudaError_t direct_adjoint_t(Plan& p, const void* r, cudaStream_t st, bool pairs = false) {
    using C = C_t<T>;
    if (p.direct_ranges.empty()) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(p.d_cdir, 0, p.N * sizeof(C), st);
    if (e != cudaSuccess) return e;
    const bool dbl = sizeof(T) == 8;
    const std::vector<DirectAdjItem>& items = dbl ? p.dadj_work64 : p.dadj_work32;
    const DirectAdjItem* d_items = dbl ? p.d_dadj64 : p.d_dadj32;
    int slot;
    timer_begin(p, "direct_adj", 0.0, st, &slot);
    const int64_t nbig = (int64_t)items.size() - p.n_dadj_small;
    if (nbig > 0 && pairs) {
        k_direct_adj_ff<<<(unsigned)nbig, 32, 0, st>>>(d_items, p.d_bands, p.d_ws, p.d_perm,
                                                      (const double2*)r, (double2*)p.d_cdir);
        ++p.launches;
    } else if (nbig > 0) {
        k_direct_adj<T><<<(unsigned)nbig, 32, 0, st>>>(d_items, p.d_bands, p.d_ws, p.d_ntab, p.d_perm,
                                                       (const C*)r, (C*)p.d_cdir);
        ++p.launches;
    }
    if (p.n_dadj_small > 0) {
        k_direct_adj_small<T><<<(unsigned)p.n_dadj_small, 32, 0, st>>>(
            d_items + nbig, p.d_bands, p.d_ws, p.d_ntab, p.d_perm, (const C*)r, (C*)p.d_cdir);
        ++p.launches;
    }
    timer_end(p, slot, st);
    return cudaGetLastError();
}

// (the float-pair form on its complex128 r: bands with K <= kDirSmallK in double)
cudaError_t run_direct_adjoint(Plan& p, const void* r, cudaStream_t st) {
    if (p.prec == FL_FP64_FF) return direct_adjoint_t<double>(p, r, st, true);
    return p.prec == FL_FP64 ? direct_adjoint_t<double>(p, r, st) : direct_adjoint_t<float>(p, r, st);
}

}  // namespace fl
