// fl_plan.cuh -- host-side plan object and the kernel launchers shared by the
// translation units of libfl.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fl.h"
#include "fl_common.cuh"

namespace fl {

constexpr int kMaxQ = 40;
constexpr int kMaxMw = 16;
constexpr int kSmallMaxLog2 = 12;   // grids up to 4096 points: one CTA per FFT
constexpr int kMaxLog2n = 24;       // two passes of <= 4096 points each

// Work item of the small-grid FFT kernel: FFTs nfft (one per right-hand side
// s0 .. s0+nfft-1) of band `band`, all of length 2^log2n.
struct SmallWork {
    int band;
    int s0;
    int nfft;
    int log2n;
};

// Thread budgets per CTA of the two passes (float / double).  Several CTAs per
// SM, so that one CTA's loads overlap the others' shared-memory stages; FP32
// pass 2 at 256 threads (4 rows of 1024 per CTA, four CTAs per SM) measured
// 2 % faster than at 512.
#ifndef FL_P1_THREADS_F32
#define FL_P1_THREADS_F32 1024
#endif
#ifndef FL_P2_THREADS_F32
#define FL_P2_THREADS_F32 256
#endif
#ifndef FL_P1_THREADS_F64
#define FL_P1_THREADS_F64 512
#endif
#ifndef FL_P2_THREADS_F64
#define FL_P2_THREADS_F64 512
#endif
// Columns (pass 1) or rows (pass 2) per CTA: up to seg contiguous bytes per
// global row segment within the thread budget TMAX (L/16 threads per FFT);
// csize = bytes per complex element.  Also used on the host (fused gather).
// Pass 1 writes whole 128-byte lines of the intermediate (FL_P1_SEG_BYTES;
// measured at N = M = 2^20 FP32: 0.593 ms against 0.635 at 64 bytes, 0.79 at
// 32 and 0.65 at 256); pass 2 keeps 64 (its row blocks fix the fused gather's
// entries).
#ifndef FL_P1_SEG_BYTES
#define FL_P1_SEG_BYTES 128
#endif
__host__ __device__ constexpr int pass_tiles(int csize, int log2L, int tmax, int seg = 64) {
    const int per = (1 << log2L) / 16;                   // threads per FFT
    const int w0 = seg / csize;
    const int wmin = (32 / per > w0) ? 32 / per : w0;    // >= one warp
    return (wmin * per <= tmax) ? wmin : tmax / per;
}

// One (band, right-hand side) of a four-step FFT launch, with the offset of
// its slice of the intermediate buffer.
struct PassItem {
    int band;
    int rhs;
    int64_t y_off;
};

// A launch of the two four-step passes over items[start, start + count), all
// of grid length 2^log2n.
struct PassGroup {
    int start, count, log2n;
};

// Device tables of the window gather fused into pass 2 (see k_pass2): per
// fused band, row-block starts into its entry list; per entry {slot, l1} (the
// node's partial-sum slot and the grid column of its taps) and the window
// values of the tile's rows (zero where the window has no tap), in float4
// groups; and the partial sums the passes write.
struct FuseArgs {
    const int32_t* rbs;
    const int2* ent;
    const float4* phi;
    float2* pp;
};

// Direct route (fl_direct.cu): kDirNodes nodes x one chunk of kDirChunk
// coefficients per CTA (its 8 warps take kDirNodes / 8 nodes each, so the
// staged chunk serves them all), Horner blocks of kDirBlock terms.
#ifndef FL_DIR_NODES
#define FL_DIR_NODES 16
#endif
constexpr int kDirBlock = 32;
constexpr int kDirChunk = 4096;
constexpr int kDirNodes = FL_DIR_NODES;
static_assert(kDirNodes % 8 == 0, "whole nodes per warp");
// below this many direct items (8 CTAs per SM of the 152) a plan halves the
// nodes per item
constexpr int64_t kDirFewItems = 8 * 152;
// FP32 bands with K <= kDirSmallK and at least kDirSmallMinNodes nodes: one
// thread per node, up to kDirSmallNodes nodes per CTA, all K terms per thread
// (see k_direct_small).  Fewer nodes, or FP64 (whose serial chains are long),
// keep a warp per node.
#ifndef FL_DIR_SMALL_MIN_NODES
#define FL_DIR_SMALL_MIN_NODES 128
#endif
#ifndef FL_DIR_SMALL_NODES
#define FL_DIR_SMALL_NODES 256
#endif
constexpr int kDirSmallK = 256, kDirSmallNodes = FL_DIR_SMALL_NODES,
              kDirSmallMinNodes = FL_DIR_SMALL_MIN_NODES;

struct DirectItem {
    int band;
    int chunk;
    int64_t node0;   // first sorted node of the item
    int nnodes;      // <= kDirNodes
    int pad;
};

// Direct route adjoint: a warp per (band, frequency chunk of 32 KL, node group).
constexpr int kDirAdjNodes = 256;
struct DirectAdjItem {
    int band;
    int kchunk;
    int64_t node0;
    int nnodes;
    int pad;
};

struct DirectRange {
    int band;
    int pad;
    int64_t count;   // nodes of the band
    int64_t prefix;  // direct nodes of the bands before it
};

// Per-band plan data on the host.
struct BandHost {
    int ell = 0, Lm = 0;    // l_m, L_m (Definition 3.2); 0 for the Y_M band
    int inst = 0;           // transform of the batch the band belongs to
    int local = 0;          // band index within its transform (0 = Z^0, 1..levels)
    int64_t nodes = 0;      // nodes of the band
    int64_t node_off = 0;   // first node of the band in sorted order
    int64_t fentries = 0;   // entries of the fused gather (0: not fused)
    BandDev dev{};
};

// One transform of a plan (a single plan has one; a batched plan has many).
// Its bands occupy bands[band_base .. band_base + levels] of the plan.
struct Instance {
    int64_t N = 0, M = 0;
    int64_t noff = 0, moff = 0;   // offsets of its coefficients and nodes/results
    int64_t src_off = 0;          // first row of its nodes in the caller's array
    int twin = -1;                // an earlier transform with the same N and nodes
    int band_base = 0;
    int levels = 1;
    double xi1 = 0;
    int64_t z0_nodes = 0;
};

struct Timer {
    std::string name;
    cudaEvent_t start, stop;
    double bytes;
};

struct Plan {
    int kind = 0;           // 0 Fourier-Laplace, 1 Laplace
    fl_precision prec = FL_FP32;
    int64_t N = 0, M = 0;
    int q = 0, levels = 1, mw = 0;
    double eps = 0, eps_K = 0, eps_A = 0, y1 = 0, xi1 = 0, kb_b = 0;
    std::vector<BandHost> bands;          // per transform: Z^0, 1..levels (see Instance)
    std::vector<Instance> inst;
    bool batched = false;
    int64_t z0_nodes = 0;
    int64_t grid_elems = 0, D_elems = 0, Y_elems = 0;
    std::vector<SmallWork> small_work;
    std::vector<int> large_bands;
    std::vector<PassItem> pass_items;
    std::vector<PassGroup> pass_groups;
    int rhs_per_launch = 0;        // four-step items per launch (0 = a whole size class)
    int fuse_mode = 0;             // window gather in pass 2: 0 by cost, 1 never, 2 wherever possible
    int sigma_mode = 0;            // oversampling: 0 by cost, 1 sigma = 2, 2 sub-bands wherever allowed
    double sigma_min = 2.0;        // smallest oversampling of the plan's grids
    int route_mode = 0;            // 0 by cost, 1 all NFFT, 2 all direct
    int variant = 0;               // 0 Algorithm 2 weights, 1 one-sided interpolation
    // real exponents xi_k >= 1 (fl_plan_xi): the Fourier factor is an NNFFT
    bool xi_mode = false;
    std::vector<double> h_xis;     // exponents in ascending order (host)
    double* d_xis = nullptr;       // the same on the device
    int32_t* d_xperm = nullptr;    // sorted position -> coefficient index
    int32_t* d_xbk = nullptr;      // floor(2 xi_k) per sorted position
    int32_t* d_xstart = nullptr;   // first sorted position with floor(2 xi) >= B, B = 0 .. 2 xi_1 + 1
    void* d_xwin = nullptr;        // frequency-window taps per sorted position (2 m_w, T)
    void* d_xiphi = nullptr;       // 1 / Phi of every NNFFT grid size (T)
    void* d_xcs = nullptr;         // coefficients in sorted exponent order (complex T, per execute)
    int2* d_xsb = nullptr;         // NNFFT bands of the spreading launch: {first block, band}
    int xsb_n = 0;                 // entries of d_xsb
    int64_t xsb_blocks = 0;        // blocks of the spreading launch
    int xqc = 0;                   // right-hand sides per spreading chunk (4, 8, 12 or 16)
    int64_t xiphi_elems = 0;
    double direct_bias = 1.0;
    double tuned_bias = 0.0;       // bias chosen by the autotuner (0: not tuned)
    int tuned_sigma_mode = -1, tuned_fuse_mode = -1, tuned_rhs = -1;   // its other choices
    std::vector<DirectItem> direct_work;   // items of the larger-K bands, then n_direct_small
    int64_t n_direct_small = 0;            // items of the bands with K <= kDirSmallK (at the end)
    std::vector<DirectRange> direct_ranges;
    std::vector<DirectAdjItem> dadj_work32, dadj_work64;   // adjoint items for KL = 32 / 16, then
    int64_t n_dadj_small = 0;                              // the items of K <= kDirSmallK bands
    int64_t direct_nodes = 0, direct_terms = 0, dpart_elems = 0;

    // device memory
    double2* d_ws = nullptr;       // nodes in sorted order (Re w, Im w)
    int32_t* d_perm = nullptr;     // sorted position -> original index
    int32_t* d_bandid = nullptr;   // band (global index) of each sorted node
    int32_t* d_cell = nullptr;     // grid cell floor(n_m x) of each sorted node
    uint4* d_ntab = nullptr;       // FP32 plans: per sorted node x 2^64 (64-bit fixed point) and
                                   // the barycentric tau of its band as a float pair
    void* d_sp_phi = nullptr;      // adjoint: window taps per node (M x 2 m_w, T)
    void* d_sp_L = nullptr;        // adjoint: barycentric weights per node (M x q, T)
    void* d_sp_rv = nullptr;       // adjoint: shifted residual per node (M, complex T)
    struct CellBand {              // adjoint: the cells of one NFFT band
        int band;
        int pad;
        int64_t prefix;            // cells of the NFFT bands before it
    };
    std::vector<CellBand> cell_bands;   // sparse bands first, then dense ones
    CellBand* d_cell_bands = nullptr;
    int n_sparse_cb = 0;
    int64_t cells_total = 0;            // cells of the sparse bands
    int64_t cells_dense = 0;            // cells of the dense bands
    BandDev* d_bands = nullptr;    // levels + 1 descriptors
    SmallWork* d_small = nullptr;
    PassItem* d_pass = nullptr;
    double* d_cheb = nullptr;      // t_s (q), lambda_s (q)
    float* d_cheb32 = nullptr;     // t_s as (hi, lo) float pairs, lambda_s in float, and the
                                   // low part of lambda_s (4 q)
    void* d_D = nullptr;           // weight tables (T)
    void* d_grid = nullptr;        // band grids (complex T)
    void* d_Y = nullptr;           // four-step intermediate (complex T)
    void* d_tw = nullptr;          // four-step stage twiddles (complex T, kTwEntries;
                                   // float pairs: + 8192 pass-1 output twiddles)
    void* d_stage_c = nullptr;     // staging for fl_execute_host and fl_execute_batched_ptrs
    void* d_stage_f = nullptr;
    int64_t* d_boff = nullptr;     // batched: instance offsets of c (B + 1) then of f (B + 1)
    void** d_bptr = nullptr;       // batched: the caller's c pointers (B) then f pointers (B)
    void* d_stage_r = nullptr;     // fl_transposed: conj of the node values
    void* d_cff = nullptr;         // FL_FP64_FF: the coefficients as float pairs (N)
    void* d_z0 = nullptr;          // one complex: sum of r over Z^0 (adjoint)
    DirectItem* d_direct = nullptr;
    DirectRange* d_dranges = nullptr;
    DirectAdjItem* d_dadj32 = nullptr;
    DirectAdjItem* d_dadj64 = nullptr;
    void* d_dpart = nullptr;       // direct route: partial sums (complex T)
    void* d_cdir = nullptr;        // direct route adjoint: N complex
    // fused gather (FuseArgs): row-block starts, entries, window values, partial sums
    int32_t* d_frbs = nullptr;
    int2* d_fent = nullptr;
    float4* d_fphi = nullptr;
    float2* d_fpp = nullptr;
    int64_t fused_bands = 0, fused_entries = 0;
    double scratch_bytes = 0;

    // Laplace (Algorithm 1)
    double* d_t = nullptr;
    double* d_s = nullptr;
    uint8_t* d_tband = nullptr;    // band of every t_k
    double* d_ts = nullptr;        // the t_k in band order (stable), for the moments
    uint8_t* d_tbs = nullptr;      // their bands
    int32_t* d_tperm = nullptr;    // original index of the k-th t in band order
    uint8_t* d_sband = nullptr;    // band of every s_j
    void* d_lap = nullptr;         // moments and partial sums
    double* d_lapK = nullptr;      // coupling blocks K^{Y_m, Omega_l} (plan-time table)
    int64_t* d_lapKoff = nullptr;  // offset of band m's blocks in d_lapK
    int lap_blocks = 0;
    int lap_kernel = 0;            // 0 Algorithm 1 (exp), 1 generalised exp, 2 generalised K_1/2
    int32_t* d_nearT = nullptr;    // generalised Algorithm 1: the t_k in Omega_M
    int64_t n_nearT = 0;

    // CUDA-graph replay of fl_execute / fl_execute_batched
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;
    const void* g_c = nullptr;
    void* g_f = nullptr;
    cudaStream_t g_st = nullptr;
    int64_t graph_launches = 0;

    // timing
    bool timing = false;
    std::vector<Timer> timers;
    int64_t launches = 0;
    double model_bytes = 0;

    ~Plan();
};

// Launchers (fl_nodes.cu).  For transform `in` of the plan: classify its M
// nodes (keys: local band << 25 | grid cell), sort, and write its slice of the
// sorted node arrays with global band ids and result indices.
cudaError_t launch_classify(const Plan& p, const Instance& in, const double* nodes, uint32_t* keys,
                            int32_t* vals, int64_t* counts, int* flag, cudaStream_t st);
cudaError_t radix_sort_pairs(uint32_t* keys, int32_t* vals, uint32_t* keys_tmp,
                             int32_t* vals_tmp, uint32_t* hist, int64_t n, int key_bits,
                             cudaStream_t st);
cudaError_t launch_permute(Plan& p, const Instance& in, const double* nodes, const uint32_t* keys,
                           const int32_t* vals, cudaStream_t st);
cudaError_t launch_copy_sorted(Plan& p, const Instance& in, const Instance& twin, cudaStream_t st);
// cell[off .. off + n) >>= shift (node cells of a band moved to a grid 2^shift times smaller)
cudaError_t launch_cell_shift(int32_t* cell, int64_t off, int64_t n, int shift, cudaStream_t st);

// Launchers (fl_transform.cu)
cudaError_t build_tables(Plan& p, const Instance& in, cudaStream_t st);
cudaError_t build_node_table(Plan& p, cudaStream_t st);   // d_ntab (FP32 forward gather)
cudaError_t build_cheb(Plan& p, cudaStream_t st);
cudaError_t build_twiddles(Plan& p, cudaStream_t st);
// rmul != nullptr: f[j] = rmul[j] * conj(result_j) (the node-gradient epilogue)
cudaError_t run_forward(Plan& p, const void* c, void* f, bool deriv, cudaStream_t st,
                        const void* rmul = nullptr);
cudaError_t run_adjoint(Plan& p, const void* r, void* c_out, cudaStream_t st);
cudaError_t run_transposed(Plan& p, const void* g, void* out, cudaStream_t st);
// Real exponents (fl_xi.cu): plan-time tables and the forward transform
cudaError_t build_xi_tables(Plan& p, cudaStream_t st);
cudaError_t launch_xi_spread(Plan& p, const void* c, cudaStream_t st);
cudaError_t launch_xi_combine(Plan& p, void* out, cudaStream_t st);   // adjoint: grids -> c
cudaError_t run_forward_xi(Plan& p, const void* c, void* f, cudaStream_t st);

// Launchers (fl_direct.cu)
cudaError_t run_direct_forward(Plan& p, const void* c, void* f, bool deriv, const void* rmul,
                               cudaStream_t st);
cudaError_t run_direct_adjoint(Plan& p, const void* r, cudaStream_t st);

// Launchers (fl_laplace.cu)
cudaError_t run_laplace(Plan& p, const void* c, void* f, cudaStream_t st);

// Per-thread error message of the C ABI (fl_api.cu)
fl_status set_error(fl_status s, const std::string& msg);
void clear_error();

// Timing helpers (fl_api.cu)
void timer_begin(Plan& p, const char* name, double bytes, cudaStream_t st, int* slot);
void timer_end(Plan& p, int slot, cudaStream_t st);

}  // namespace fl

// The opaque handle of include/fl.h.
struct fl_plan_s {
    fl::Plan p;
};
