// fl_nodes.cu -- node preparation for Algorithm 2 (Kunis & Melzer, Section 4):
// polar split z = exp(-y) exp(2 pi i x) (eq. 4.2), removal of Z^0 = {|z| < eps},
// assignment of every node to its dyadic band Y_m (Definition 3.2), and a
// stable LSD radix sort of the nodes by (band, grid cell) so that the gather
// of each band reads its grid in order.
#include "fl_plan.cuh"

namespace fl {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Band index of v in [0, v1]: v in (v1/2^b, v1/2^(b-1)] -> b for b < levels,
// v <= v1/2^(levels-1) -> levels.  All comparisons are against exact power-of-two
// scalings of v1, so the assignment is exact.
__device__ __forceinline__ int band_of(double v, double v1, int levels) {
    if (levels <= 1) return 1;
    if (v > ldexp(v1, -1)) return 1;
    if (!(v > ldexp(v1, -(levels - 1)))) return levels;
    int b = (int)floor(log2(v1 / v)) + 1;
    b = max(1, min(b, levels - 1));
    while (b > 1 && v > ldexp(v1, -(b - 1))) --b;
    while (b < levels - 1 && !(v > ldexp(v1, -b))) ++b;
    return b;
}

// xhalf (real exponents): the grid coordinate is x/2 (the NNFFT's outer NFFT
// runs at x/2) and |Re w| <= 1/2 is required (principal branch of z^xi).
__global__ void k_classify(int64_t M, const double* __restrict__ w,
                           const BandDev* __restrict__ bands, int levels, double y1,
                           int constant_only, int xhalf, uint32_t* __restrict__ keys,
                           int32_t* __restrict__ vals, unsigned long long* __restrict__ counts,
                           int* __restrict__ flag) {
    __shared__ unsigned int cnt[FL_MAX_LEVELS + 1];
    for (int i = threadIdx.x; i <= FL_MAX_LEVELS; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < M) {
        const double x = w[2 * j], v = w[2 * j + 1];
        int band = 0;
        uint32_t cell = 0;
        if (!(v >= 0.0) || !isfinite(x) || !isfinite(v) || (xhalf && !(fabs(x) <= 0.5))) {
            atomicOr(flag, 1);
        } else if (!constant_only) {
            const double y = kTwoPi * v;          // the paper's radial variable
            band = (y > y1) ? 0 : band_of(y, y1, levels);
            const int64_t n = bands[band].n;
            if (band > 0 && n > 0) {
                const double xs = xhalf ? 0.5 * x : x;   // exact
                const double xr = xs - floor(xs);        // exact
                cell = (uint32_t)floor(xr * (double)n);  // exact: n is a power of two
            }
        }
        keys[j] = ((uint32_t)band << 25) | cell;
        vals[j] = (int32_t)j;
        atomicAdd(&cnt[band], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= levels; i += blockDim.x)
        if (cnt[i]) atomicAdd(&counts[i], (unsigned long long)cnt[i]);
}

cudaError_t launch_classify(const Plan& p, const Instance& in, const double* nodes, uint32_t* keys,
                            int32_t* vals, int64_t* counts, int* flag, cudaStream_t st) {
    if (in.M == 0) return cudaSuccess;
    const int bs = 256;
    const int64_t grid = (in.M + bs - 1) / bs;
    k_classify<<<(unsigned)grid, bs, 0, st>>>(in.M, nodes + 2 * in.src_off, p.d_bands + in.band_base,
                                              in.levels, p.y1, (in.N == 1 && !p.xi_mode) ? 1 : 0,
                                              p.xi_mode ? 1 : 0, keys, vals,
                                              (unsigned long long*)(counts + in.band_base), flag);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) pairs, 8-bit digits.

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void k_rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                          uint32_t* __restrict__ hist, int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = tile + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `total` counters by one block of 1024 threads.
__global__ void k_rs_scan(uint32_t* __restrict__ hist, int64_t total) {
    __shared__ uint32_t part[1024];
    const int64_t chunk = (total + 1023) / 1024;
    const int64_t lo = threadIdx.x * chunk;
    const int64_t hi = min(total, lo + chunk);
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += hist[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;   // exclusive prefix of this chunk
    for (int64_t i = lo; i < hi; ++i) {
        const uint32_t v = hist[i];
        hist[i] = run;
        run += v;
    }
}

__global__ void k_rs_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                             uint32_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                             int shift, const uint32_t* __restrict__ offs, int nblocks) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[RS_THREADS / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    base[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
    const int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < RS_ITEMS; ++r) {
        for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const int64_t i = tile + r * RS_THREADS + tid;
        const bool valid = i < n;
        uint32_t key = 0;
        int32_t val = 0;
        unsigned d = 256;   // sentinel for lanes past the end
        if (valid) {
            key = kin[i];
            val = vin[i];
            d = (key >> shift) & 255u;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = base[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < RS_THREADS / 32; ++w) add += wcnt[w][tid];
        base[tid] += add;
        __syncthreads();
    }
}

cudaError_t radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_tmp,
                             int32_t* vals_tmp, uint32_t* hist, int64_t n, int key_bits,
                             cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    const int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
    uint32_t *ka = keys, *kb = keys_tmp;
    int32_t *va = vals, *vb = vals_tmp;
    int passes = 0;
    for (int shift = 0; shift < key_bits; shift += 8, ++passes) {
        k_rs_hist<<<nblocks, RS_THREADS, 0, st>>>(ka, n, shift, hist, nblocks);
        k_rs_scan<<<1, 1024, 0, st>>>(hist, (int64_t)256 * nblocks);
        k_rs_scatter<<<nblocks, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, hist, nblocks);
        uint32_t* tk = ka; ka = kb; kb = tk;
        int32_t* tv = va; va = vb; vb = tv;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (passes & 1) {   // result sits in the temporaries: copy back
        e = cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    }
    return e;
}

// Sorted slice of one transform: node (Re w, Im w), result index moff + j and
// global band id band_base + local band.
__global__ void k_permute(int64_t M, const double* __restrict__ w, const uint32_t* __restrict__ keys,
                          const int32_t* __restrict__ vals, int32_t moff, int32_t band_base,
                          double2* __restrict__ ws, int32_t* __restrict__ perm,
                          int32_t* __restrict__ bandid, int32_t* __restrict__ cell) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int32_t j = vals[i];
    ws[i] = make_double2(w[2 * (int64_t)j], w[2 * (int64_t)j + 1]);
    perm[i] = moff + j;
    bandid[i] = band_base + (int32_t)(keys[i] >> 25);
    cell[i] = (int32_t)(keys[i] & ((1u << 25) - 1u));
}

cudaError_t launch_permute(Plan& p, const Instance& in, const double* nodes, const uint32_t* keys,
                           const int32_t* vals, cudaStream_t st) {
    if (in.M == 0) return cudaSuccess;
    const int bs = 256;
    k_permute<<<(unsigned)((in.M + bs - 1) / bs), bs, 0, st>>>(
        in.M, nodes + 2 * in.src_off, keys, vals, (int32_t)in.moff, in.band_base, p.d_ws + in.moff,
        p.d_perm + in.moff, p.d_bandid + in.moff, p.d_cell + in.moff);
    return cudaGetLastError();
}

// A transform whose nodes and N equal an earlier one's (shared node sets)
// takes that transform's sorted slice: the same order and cells, its own
// result indices and band ids.
__global__ void k_copy_sorted(int64_t M, const double2* __restrict__ ws_src,
                              const int32_t* __restrict__ perm_src, const int32_t* __restrict__ band_src,
                              const int32_t* __restrict__ cell_src, int32_t dm, int32_t db,
                              double2* __restrict__ ws, int32_t* __restrict__ perm,
                              int32_t* __restrict__ bandid, int32_t* __restrict__ cell) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    ws[i] = ws_src[i];
    perm[i] = perm_src[i] + dm;
    bandid[i] = band_src[i] + db;
    cell[i] = cell_src[i];
}

cudaError_t launch_copy_sorted(Plan& p, const Instance& in, const Instance& twin, cudaStream_t st) {
    if (in.M == 0) return cudaSuccess;
    const int bs = 256;
    k_copy_sorted<<<(unsigned)((in.M + bs - 1) / bs), bs, 0, st>>>(
        in.M, p.d_ws + twin.moff, p.d_perm + twin.moff, p.d_bandid + twin.moff, p.d_cell + twin.moff,
        (int32_t)(in.moff - twin.moff), in.band_base - twin.band_base, p.d_ws + in.moff,
        p.d_perm + in.moff, p.d_bandid + in.moff, p.d_cell + in.moff);
    return cudaGetLastError();
}

__global__ void k_cell_shift(int32_t* __restrict__ cell, int64_t n, int shift) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cell[i] >>= shift;
}

// floor(x n) >> s = floor(x n / 2^s) for the power-of-two grid sizes n: the
// cells of the smaller grid, and the sorted order is kept.
cudaError_t launch_cell_shift(int32_t* cell, int64_t off, int64_t n, int shift, cudaStream_t st) {
    if (n == 0 || shift == 0) return cudaSuccess;
    k_cell_shift<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cell + off, n, shift);
    return cudaGetLastError();
}

}  // namespace fl
