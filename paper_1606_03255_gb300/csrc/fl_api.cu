// fl_api.cu -- the C ABI of libfl.so (include/fl.h): parameter selection
// (Definition 3.2 and Algorithm 2 of Kunis & Melzer), band sizing, plan
// construction, execution, timing and error reporting.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "fl_plan.cuh"

namespace fl {

static thread_local std::string g_err;

fl_status set_error(fl_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

void clear_error() { g_err.clear(); }

static fl_status fail(fl_status s, const std::string& msg) { return set_error(s, msg); }

static fl_status cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FL_ENOMEM : FL_ECUDA;
}

#define FL_CUDA(call, where)                          \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

Plan::~Plan() {
    if (gexec) cudaGraphExecDestroy(gexec);
    void* ptrs[] = {d_ws, d_perm, d_bandid, d_bands, d_small, d_pass, d_cheb, d_D, d_grid, d_Y,
                    d_stage_c, d_stage_f, d_stage_r, d_z0, d_t, d_s, d_tband, d_sband, d_lap, d_direct,
                    d_dranges, d_dpart, d_cdir, d_dadj32, d_dadj64, d_cell, d_sp_phi,
                    d_sp_L, d_sp_rv, d_cell_bands, d_lapK, d_lapKoff, d_tw, d_nearT, d_cheb32, d_cff, d_tperm, d_ts, d_tbs,
                    d_xis, d_xperm, d_xbk, d_xstart, d_xwin, d_xiphi, d_xcs, d_xsb,
                    d_frbs, d_fent, d_fphi, d_fpp, d_ntab, d_boff, d_bptr};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (Timer& t : timers) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
}

void timer_begin(Plan& p, const char* name, double bytes, cudaStream_t st, int* slot) {
    *slot = -1;
    if (!p.timing) return;
    Timer t;
    t.name = name;
    t.bytes = bytes;
    if (cudaEventCreate(&t.start) != cudaSuccess) return;
    if (cudaEventCreate(&t.stop) != cudaSuccess) {
        cudaEventDestroy(t.start);
        return;
    }
    cudaEventRecord(t.start, st);
    p.timers.push_back(t);
    *slot = (int)p.timers.size() - 1;
}

void timer_end(Plan& p, int slot, cudaStream_t st) {
    if (slot >= 0) cudaEventRecord(p.timers[slot].stop, st);
}

static int ilog2_ceil(int64_t v) {
    int l = 0;
    while (((int64_t)1 << l) < v) ++l;
    return l;
}

// Smallest Kaiser-Bessel half-width m whose aliasing-plus-truncation estimate
// 4 pi (sqrt(m) + m) (1 - 1/sigma)^(1/4) exp(-2 pi m sqrt(1 - 1/sigma))
// (the error bound of the Kaiser-Bessel NFFT) is at most eps.
static int window_width(double eps, double sigma) {
    const double a = sqrt(1.0 - 1.0 / sigma);
    for (int m = 2; m <= 12; ++m) {
        const double bound = 4.0 * M_PI * (sqrt((double)m) + m) * sqrt(a) * exp(-2.0 * M_PI * m * a);
        if (bound <= eps) return m;
    }
    return 12;
}

// Parameters of Algorithm 2 (Section 4) with the error split of Lemma 4.1 that
// do not depend on N: q, y_1 = ln(1/eps), the window.
// One-sided interpolation rank: the smallest q whose per-entry bound
// max_k |exp(-y k) - sum_s L_s(y) exp(-y_s k)| <= 2 q^q e^-q / (4^q q!) on a
// band (a, 2a] is at most eps_K.  The bound is the interpolation error formula
// of Section 2 with diam = a and max |d^q/dy^q exp(-y k)| = k^q exp(-a k),
// maximised over k a = q.
static int onesided_rank(double eps_K) {
    for (int q = 1; q <= kMaxQ; ++q) {
        const double lb = log(2.0) + q * log((double)q) - q - q * log(4.0) - lgamma(q + 1.0);
        if (lb <= log(eps_K)) return q;
    }
    return kMaxQ + 1;
}

static fl_status select_common(Plan& p, int q_in) {
    p.eps_K = p.eps / 3.0;
    p.eps_A = p.eps / 3.0;
    if (q_in > 0)
        p.q = q_in;
    else if (p.variant == 1)
        p.q = onesided_rank(p.eps_K);
    else
        p.q = (int)ceil(0.5 + log(1.0 / p.eps_K) / log(4.0));
    if (p.q > kMaxQ) return fail(FL_EUNSUPPORTED, "interpolation rank q above 40");
    p.y1 = log(1.0 / p.eps);            // Z^0 removed: y in [0, ln(1/eps)]
    // real exponents: two windows (frequency spreading and the outer NFFT),
    // the latter's error amplified by up to Phi(0)/Phi(1/4) < 8 in the division
    // by Phi(x/2): each gets eps_A / 8
    p.mw = window_width(p.xi_mode ? p.eps_A / 8.0 : p.eps_A, 2.0);
    p.kb_b = M_PI * (2.0 - 1.0 / 2.0);
    return FL_OK;
}

// Real exponents: Definition 3.2 with xi_1 = max xi_k; band m keeps the sorted
// exponents xi_k <= xi_1 / 2^(l_m - 1) (a prefix of length K).  Its NNFFT
// spreads them, centred on xc (2 xc = floor(xi_min + cut), an integer), onto the
// frequency grid of spacing 1/2 (grid frequency g <-> xi = xc + g/2; taps
// g in (2(xi - xc) - m_w, 2(xi - xc) + m_w]); the occupied |g| <= gh, and the
// outer NFFT has bandwidth Nm = 2^lg >= 2 gh + 2 on n = 2 Nm points.  The
// dyadic cuts lie just below powers of two, so the window margin m_w + 1 alone
// would double Nm; the half-size Nm is kept when it misses at most m_w + 3
// occupied frequencies, e = gh - (Nm/2 - 1), and these raise the
// Kaiser-Bessel aliasing term by at most 1 %: the nearest alias of frequency
// Nm/2 - 1 + e sits at |nu| = 3/4 - e/n, where Phi = pi I_0(m_w pi sqrt(6 e / n))
// (b = 3 pi / 2), so the condition is m_w pi sqrt(6 e / n) <= 0.2 (I_0(0.2) = 1.01).
static fl_status select_bands_xi(Plan& p, Instance& in, int inst_index) {
    const std::vector<double>& xs = p.h_xis;
    in.xi1 = xs.empty() ? 0.0 : xs.back();
    const double lv = ceil(log2(p.y1 * in.xi1 / p.eps_K)) + 1.0;
    in.levels = (int)std::max(1.0, lv);
    if (in.levels > 127) return fail(FL_EUNSUPPORTED, "more than 127 dyadic levels");
    in.band_base = (int)p.bands.size();
    for (int b = 0; b <= in.levels; ++b) {
        BandHost bh;
        bh.inst = inst_index;
        bh.local = b;
        bh.dev.c_off = in.noff;
        bh.dev.parent = -1;
        bh.dev.kb = p.kb_b;
        if (b == 0) {
            p.bands.push_back(bh);
            continue;
        }
        double cut = in.xi1;
        if (b < in.levels) {
            const double lg = log2(p.y1 * in.xi1) - b - log2(log(1.0 / p.eps_K));
            bh.ell = std::max(1, (int)floor(lg) + 1);
            bh.Lm = in.levels - b;
            cut = std::min(in.xi1, ldexp(in.xi1, 1 - bh.ell));
            bh.dev.nrhs = p.q;
            const double a = ldexp(p.y1, -b);
            bh.dev.yc = 1.5 * a;
            bh.dev.yh = 0.5 * a;
            bh.dev.yh_inv = 1.0 / bh.dev.yh;
        } else {
            bh.dev.nrhs = 1;
        }
        const int64_t K = (int64_t)(std::upper_bound(xs.begin(), xs.end(), cut) - xs.begin());
        const double lo = K > 0 ? xs[0] : cut;
        const double two_xc = floor(lo + cut);
        bh.dev.xc = 0.5 * two_xc;
        bh.dev.gh = (int64_t)std::max(ceil(two_xc - 2.0 * lo), ceil(2.0 * cut - two_xc)) + p.mw + 1;
        int lg = std::max(4, ilog2_ceil(2 * bh.dev.gh + 2));
        if (lg > 4) {
            const int64_t e = bh.dev.gh - (((int64_t)1 << (lg - 1)) / 2 - 1);
            if (e <= p.mw + 3 && p.mw * M_PI * sqrt(6.0 * (double)e / ldexp(1.0, lg)) <= 0.2) --lg;
        }
        bh.dev.K = K;
        bh.dev.Nm = (int64_t)1 << lg;
        bh.dev.log2n = lg + 1;
        bh.dev.n = (int64_t)1 << (lg + 1);
        if (bh.dev.log2n > kMaxLog2n) return fail(FL_EUNSUPPORTED, "NNFFT grid above 2^24 points");
        p.bands.push_back(bh);
    }
    return FL_OK;
}

// Right-hand sides per chunk of the real-exponent spreading, QC in {4, 8, 12,
// 16}: each chunk passes over a grid frequency's exponents once, at about
// 10 + QC/4 + 2 QC instructions per exponent (index, window and coefficient;
// the 16-byte weight loads; the complex multiply-adds), the last chunk padded
// with zero weights.  The QC of least total cost for q.
static int xi_chunk(int q) {
    int best = 4, best_cost = 1 << 30;
    for (int qc : {16, 12, 8, 4}) {
        const int cost = (q + qc - 1) / qc * (10 + qc / 4 + 2 * qc);
        if (cost < best_cost) {
            best = qc;
            best_cost = cost;
        }
    }
    return best;
}

// The dyadic partition of one transform (Definition 3.2 with xi_1 = N - 1):
// appends its bands 0..levels to p.bands.
static fl_status select_bands(Plan& p, Instance& in, int inst_index) {
    if (p.xi_mode) return select_bands_xi(p, in, inst_index);
    in.xi1 = (double)(in.N - 1);        // frequencies 0..N-1
    if (in.N == 1) {
        in.levels = 1;
    } else {
        const double lv = ceil(log2(p.y1 * in.xi1 / p.eps_K)) + 1.0;
        in.levels = (int)std::max(1.0, lv);
    }
    if (in.levels > 127) return fail(FL_EUNSUPPORTED, "more than 127 dyadic levels");
    in.band_base = (int)p.bands.size();
    for (int b = 0; b <= in.levels; ++b) {
        BandHost bh;
        bh.inst = inst_index;
        bh.local = b;
        bh.dev.c_off = in.noff;
        bh.dev.parent = -1;
        bh.dev.kb = p.kb_b;
        if (b == 0) {
            p.bands.push_back(bh);
            continue;
        }
        int64_t K;
        if (b < in.levels) {
            const double lg = log2(p.y1 * in.xi1) - b - log2(log(1.0 / p.eps_K));
            bh.ell = std::max(1, (int)floor(lg) + 1);
            bh.Lm = in.levels - b;
            // frequencies k <= xi1 / 2^(l_m - 1) carry weight (Lemma A.2(ii))
            K = std::min<int64_t>(in.N, (int64_t)floor(ldexp(in.xi1, 1 - bh.ell)) + 1);
            bh.dev.nrhs = p.q;
            const double a = ldexp(p.y1, -b);
            bh.dev.yc = 1.5 * a;
            bh.dev.yh = 0.5 * a;
            bh.dev.yh_inv = 1.0 / bh.dev.yh;
        } else {
            K = in.N;           // Z_M band: kernel ~ 1, one plain NFFT
            bh.dev.nrhs = 1;
        }
        const int lg = std::max(4, ilog2_ceil(K));
        bh.dev.K = K;
        bh.dev.Nm = (int64_t)1 << lg;
        bh.dev.log2n = lg + 1;
        bh.dev.n = (int64_t)1 << (lg + 1);
        if (bh.dev.log2n > kMaxLog2n) return fail(FL_EUNSUPPORTED, "grid above 2^24 points");
        p.bands.push_back(bh);
    }
    return FL_OK;
}

// Route of a non-empty band: NFFT with nrhs right-hand sides, or the direct sum
// over its K frequencies.  Costs in issued instructions: an FFT grid point
// ~ (log2 n + 8) over both passes and the prep (twice that in double, whose
// twiddles come from double sincospi); per gathered node, 2 per tap and
// right-hand side plus the window (2 m_w sinh/sqrt) and the barycentric
// divisions, both several times dearer in double on this part; a fixed launch
// and latency share per NFFT band; a direct term ~ 6 (one complex Horner step
// and its share of the block's phase).
static int route_of(const Plan& p, const BandHost& bh) {
    if (p.route_mode == 1) return 1;
    if (p.route_mode == 2) return 2;
    const BandDev& d = bh.dev;
    const bool dbl = p.prec != FL_FP32;   // float pairs: gather and direct bands in double
    const double fft_pt = dbl ? 2.0 : 1.0, win = dbl ? 150.0 : 20.0, div = dbl ? 40.0 : 4.0;
    const double per_node = (double)d.nrhs * 2 * p.mw * 2 + 2.0 * p.mw * win + (d.nrhs > 1 ? p.q * div : 0.0);
    const double fft = (double)d.nrhs * d.n * (d.log2n + 8) * fft_pt + (double)bh.nodes * per_node + 2.0e5;
    const double direct = (double)bh.nodes * d.K * 6.0 * p.direct_bias;
    return direct < fft ? 2 : 1;
}

// Four-step work items of the large bands, grouped by grid size into launches
// of at most rhs_per_launch items (0: a whole size class) and at most
// kMaxYElems intermediate elements, a band's items never split between two
// launches (a launch holding one band may exceed the cap); sets Y_elems.
constexpr int64_t kMaxYElems = (int64_t)1 << 28;

static void build_pass_groups(Plan& p) {
    p.pass_items.clear();
    p.pass_groups.clear();
    p.Y_elems = 0;
    for (int lg = kSmallMaxLog2 + 1; lg <= kMaxLog2n; ++lg) {
        const int64_t n = (int64_t)1 << lg;
        int cap = (int)std::min<int64_t>(65535, std::max<int64_t>(1, kMaxYElems / n));
        if (p.rhs_per_launch > 0) cap = std::min(cap, p.rhs_per_launch);
        int cnt = 0;
        auto close = [&]() {
            if (cnt == 0) return;
            p.pass_groups.push_back(PassGroup{(int)p.pass_items.size() - cnt, cnt, lg});
            p.Y_elems = std::max<int64_t>(p.Y_elems, (int64_t)cnt * n);
            cnt = 0;
        };
        for (int b : p.large_bands) {
            const BandDev& d = p.bands[b].dev;
            if (d.log2n != lg) continue;
            if (cnt > 0 && cnt + d.nrhs > cap) close();
            for (int s = 0; s < d.nrhs; ++s) {
                p.pass_items.push_back({b, s, (int64_t)cnt * n});
                ++cnt;
            }
        }
        close();
    }
}

// Window gather fused into pass 2 (FP32 forward, four-step grids).  A band
// qualifies when its nodes are few for its grid: per right-hand side the
// unfused path writes the grid (8 n bytes) and gathers about three 32-byte
// sectors per node, the fused one reads its entries (8 + 16 NQ bytes: slot,
// column, window values) and writes and later reads one partial sum per entry.  Each node's
// window of 2 m_w taps at grid indices lo .. lo + 2 m_w - 1 (lo = floor(n x) -
// m_w + 1, mod n) is cut into entries, one per pass-2 row block its taps fall
// in (tile rows TR of the length-n1 pass, rows l2 = g mod n2, column l1 = g /
// n2); the window values are those of the gather kernel, phi_t = kb(frac(n x)
// + m_w - 1 - t), in FP64 rounded once.
static double kb_window_host(double t, double m, double b) {
    const double s2 = m * m - t * t;
    if (!(s2 > 0.0)) return b;
    const double r = sqrt(s2);
    return sinh(b * r) / r;
}

static fl_status build_fused(Plan& p, cudaStream_t st) {
    p.fused_bands = p.fused_entries = 0;
    if (p.prec != FL_FP32 || p.xi_mode || p.fuse_mode == 1 || p.M == 0) return FL_OK;
    struct Cand {
        int b, l1, l2, TR, P;
    };
    std::vector<Cand> cands;
    const int taps = 2 * p.mw;
    for (int b = 0; b < (int)p.bands.size(); ++b) {
        BandHost& bh = p.bands[b];
        BandDev& d = bh.dev;
        d.fused = 0;
        if (d.route != 1 || d.nsub > 0 || d.log2n <= kSmallMaxLog2 || bh.nodes == 0) continue;
        const int l2 = d.log2n / 2, l1 = (d.log2n + 1) / 2;
        const int TR = pass_tiles(8, l1, FL_P2_THREADS_F32);
        const int P = (taps - 1 + TR - 1) / TR + 1;
        const int NQ = (TR + 3) / 4;
        const double parts = (double)(TR + taps - 1) / TR;
        const double unfused = 8.0 * d.n + std::min<double>(8.0 * d.n, 96.0 * bh.nodes);
        const double fused = bh.nodes * parts * (8.0 + 16.0 * NQ + 8.0) + 8.0 * P * bh.nodes;
        // sub-bands (parent >= 0) have no other gather: always fused
        if (p.fuse_mode == 2 || d.parent >= 0 || fused <= 0.5 * unfused) cands.push_back({b, l1, l2, TR, P});
    }
    if (cands.empty()) return FL_OK;
    std::vector<double2> hw(p.M);
    FL_CUDA(cudaMemcpyAsync(hw.data(), p.d_ws, p.M * sizeof(double2), cudaMemcpyDeviceToHost, st),
            "fl_plan: copy nodes");
    FL_CUDA(cudaStreamSynchronize(st), "fl_plan: synchronise");
    std::vector<int32_t> rbs;
    std::vector<int2> ent;
    std::vector<float4> phi;
    int64_t pp = 0;
    for (const Cand& cd : cands) {
        BandHost& bh = p.bands[cd.b];
        BandDev& d = bh.dev;
        const int64_t n = d.n, n2 = (int64_t)1 << cd.l2, nrb = n2 / cd.TR;
        const int NQ = (cd.TR + 3) / 4;
        struct E {
            int64_t rb;
            int slot, l1;
            float w[8];
        };
        std::vector<E> es;
        es.reserve((size_t)(bh.nodes * ((cd.TR + taps - 1) / cd.TR + 1)));
        for (int64_t jl = 0; jl < bh.nodes; ++jl) {
            const double x = hw[bh.node_off + jl].x;
            const double xr = x - floor(x);
            const double t0 = (double)n * xr;
            const double u = floor(t0);
            const double fr = t0 - u;
            const int64_t lo = (int64_t)u - (p.mw - 1);
            int part = 0;
            int64_t cur = -1;
            for (int t = 0; t < taps; ++t) {
                const int64_t g = ((lo + t) % n + n) % n;
                const int64_t rho = g & (n2 - 1);
                const int64_t rb = rho / cd.TR;
                if (rb != cur) {
                    if (part == cd.P)   // a window spans at most P row blocks (n2 >= 8 TR)
                        return fail(FL_ECUDA, "fl_plan: fused gather entry count out of range");
                    E e{};
                    e.rb = rb;
                    e.slot = (int)(jl * cd.P + part++);
                    e.l1 = (int)(g >> cd.l2);
                    es.push_back(e);
                    cur = rb;
                }
                es.back().w[rho % cd.TR] = (float)kb_window_host(fr + (double)(p.mw - 1 - t), (double)p.mw, d.kb);
            }
        }
        // bucket by row block (stable: node order within a block)
        std::vector<int32_t> cnt(nrb + 1, 0);
        for (const E& e : es) ++cnt[e.rb + 1];
        for (int64_t r = 0; r < nrb; ++r) cnt[r + 1] += cnt[r];
        d.fused = 1;
        d.pparts = cd.P;
        d.ent_off = (int64_t)ent.size();
        d.rbs_off = (int64_t)rbs.size();
        d.ph_off = (int64_t)phi.size();
        d.pp_off = pp;
        bh.fentries = (int64_t)es.size();
        rbs.insert(rbs.end(), cnt.begin(), cnt.end());
        std::vector<int32_t> pos(cnt.begin(), cnt.end() - 1);
        const size_t e0 = ent.size(), q0 = phi.size();
        ent.resize(e0 + es.size());
        phi.resize(q0 + es.size() * NQ);
        for (const E& e : es) {
            const int64_t k = pos[e.rb]++;
            ent[e0 + k] = make_int2(e.slot, e.l1);
            for (int qd = 0; qd < NQ; ++qd)
                phi[q0 + k * NQ + qd] = make_float4(e.w[4 * qd], e.w[4 * qd + 1], e.w[4 * qd + 2], e.w[4 * qd + 3]);
        }
        pp += (int64_t)d.nrhs * bh.nodes * cd.P;   // per right-hand side: one slot per (node, row block)
        ++p.fused_bands;
    }
    p.fused_entries = (int64_t)ent.size();

    FL_CUDA(cudaMalloc((void**)&p.d_frbs, rbs.size() * sizeof(int32_t)), "cudaMalloc fused starts");
    FL_CUDA(cudaMalloc((void**)&p.d_fent, ent.size() * sizeof(int2)), "cudaMalloc fused entries");
    FL_CUDA(cudaMalloc((void**)&p.d_fphi, phi.size() * sizeof(float4)), "cudaMalloc fused windows");
    FL_CUDA(cudaMalloc((void**)&p.d_fpp, pp * sizeof(float2)), "cudaMalloc fused partials");
    FL_CUDA(cudaMemcpyAsync(p.d_frbs, rbs.data(), rbs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st),
            "copy fused starts");
    FL_CUDA(cudaMemcpyAsync(p.d_fent, ent.data(), ent.size() * sizeof(int2), cudaMemcpyHostToDevice, st),
            "copy fused entries");
    FL_CUDA(cudaMemcpyAsync(p.d_fphi, phi.data(), phi.size() * sizeof(float4), cudaMemcpyHostToDevice, st),
            "copy fused windows");
    // slots beyond a node's parts are never written and must read as zero
    FL_CUDA(cudaMemsetAsync(p.d_fpp, 0, pp * sizeof(float2), st), "clear fused partials");
    // the host vectors are released on return: finish the copies first
    FL_CUDA(cudaStreamSynchronize(st), "fl_plan: synchronise");
    return FL_OK;
}

// Oversampling picked from the tolerance (FP32 forward plans).  The NFFT of a
// band with K frequencies may be computed as P NFFTs over contiguous
// sub-ranges of about K/P frequencies, each centred on its own range and
// evaluated on a power-of-two grid n >= sigma_min K_p: e.g. K = 2^20 as 3
// grids of 2^19 points (sigma = 1.5) or 5 of 2^18 (sigma = 1.25) instead of
// one of 2^21 (sigma = 2) -- linearity of A~ in its frequency columns.  The
// window half-width m_w is the smallest meeting the Kaiser-Bessel estimate at
// eps/3 for the smallest sigma used (one m_w for the plan, every band at least
// as accurate); each grid gets the window shape b = pi (2 - 1/sigma) of its
// own sigma.  Split bands always gather inside pass 2 (see build_fused), so
// only bands that qualify for that are candidates.  For each floor sigma_min
// in {2, 1.75, 1.5, 1.25} every band takes its cheapest split with sigma >=
// sigma_min by an estimate of issued instructions (FFT points x (log2 n + 8),
// fused entries and partial sums, the unfused gather's taps and window
// values, at the m_w of sigma_min); the cheapest floor wins, and m_w is then
// set for the smallest sigma it actually chose.
static double fft_cost(int nrhs, int64_t n, int log2n) { return (double)nrhs * n * (log2n + 8); }

// FP32 rounding of a band grid is amplified by the deconvolution: the weights
// 1/Phi(nu) of the highest frequency (nu = 1/(2 sigma)) exceed those of the
// lowest by Phi(0)/Phi(1/(2 sigma)) ~ exp(m_w (b - sqrt(b^2 - (pi/sigma)^2))),
// b = pi (2 - 1/sigma): about 4 at sigma = 2 (m_w = 5), 29 at sigma = 1.5
// (m_w = 6), 300 at sigma = 1.31 (m_w = 7).  Sub-bands are used only where
// it stays <= 32, the factor the FP32 error bound allows for rounding.
constexpr double kMaxDeconvGain = 32.0;

static double deconv_gain(double sigma, int mw) {
    const double b = M_PI * (2.0 - 1.0 / sigma), v = M_PI / sigma;
    return exp((double)mw * (b - sqrt(b * b - v * v)));
}

// FP64 plans: the gain times the grids' rounding, 2^6 units of 2^-53, stays
// below the NFFT's share of the tolerance (e.g. <= 47 at eps = 1e-12, so
// sigma >= 1.75 there; no practical limit at 1e-6).
static double deconv_gain_limit64(double eps_A) { return eps_A * ldexp(1.0, 47); }

static double fused_cost(int64_t nodes, int log2n, int mw) {   // per right-hand side
    const int TR = pass_tiles(8, (log2n + 1) / 2, FL_P2_THREADS_F32);
    const double entries = (double)nodes * (TR + 2 * mw - 1) / TR;
    const int parts = (2 * mw - 1 + TR - 1) / TR + 1;
    return entries * 24.0 + (double)nodes * parts * 6.0;
}

static double unfused_cost(int64_t nodes, int nrhs, int mw) {
    return (double)nodes * ((double)nrhs * 2 * mw * 2 + 2.0 * mw * 20.0);
}

struct SplitChoice {
    int P = 1, log2n = 0;
    int64_t Kp = 0, Nc = 0;
};

// Best split of band bh at sigma_min >= smin with window half-width mw
// (P = 1: unsplit); force: fewest grid points regardless of the gather.
static SplitChoice best_split(const Plan& p, const BandHost& bh, double smin, int mw, bool force,
                             double* cost) {
    const BandDev& d = bh.dev;
    SplitChoice best;
    const bool four_step = d.log2n > kSmallMaxLog2;
    // FP32: sub-bands gather inside pass 2 (fused); FP64: from their grids
    const bool fusable = p.prec == FL_FP32 && p.fuse_mode != 1;
    double c1 = fft_cost(d.nrhs, d.n, d.log2n) +
                (four_step && fusable
                     ? std::min(d.nrhs * fused_cost(bh.nodes, d.log2n, mw), unfused_cost(bh.nodes, d.nrhs, mw))
                     : unfused_cost(bh.nodes, d.nrhs, mw));
    double bc = force ? (double)d.n : c1;
    const bool eligible = smin < 2.0 && four_step && !p.xi_mode && bh.nodes > 0 &&
                          (fusable || p.prec == FL_FP64);
    const double gain_max = p.prec == FL_FP32 ? kMaxDeconvGain : deconv_gain_limit64(p.eps_A);
    // (the window shape and gain are those of the candidate's own sigma)
    if (eligible) {
        for (int P = 2; P <= 9; ++P) {
            const int64_t Kp = (d.K + P - 1) / P;
            const int64_t Nc = Kp + (Kp & 1);
            const int lg = ilog2_ceil((int64_t)ceil(smin * (double)Nc));
            if (lg <= kSmallMaxLog2 || lg > kMaxLog2n) continue;
            const int64_t n = (int64_t)1 << lg;
            if ((double)n >= 2.0 * (double)Nc) continue;   // no gain over sigma = 2
            // the half-width this sigma needs, and the FP32 limit at it
            const int mc = std::max(mw, window_width(p.eps_A, (double)n / (double)Nc));
            if (deconv_gain((double)n / (double)Nc, mc) > gain_max) continue;
            const double gather = fusable ? d.nrhs * fused_cost(bh.nodes, lg, mc) : unfused_cost(bh.nodes, d.nrhs, mc);
            const double c = force ? (double)P * n : P * (fft_cost(d.nrhs, n, lg) + gather);
            if (c < bc) {
                bc = c;
                best.P = P;
                best.log2n = lg;
                best.Kp = Kp;
                best.Nc = Nc;
            }
        }
    }
    *cost = best.P == 1 ? c1 : (force ? 0.0 : bc);
    return best;
}

static fl_status plan_splits(Plan& p, const std::vector<int>& nfft, cudaStream_t st) {
    p.sigma_min = 2.0;
    if (p.sigma_mode == 1 || p.xi_mode || p.prec == FL_FP64_FF || (p.prec == FL_FP32 && p.fuse_mode == 1))
        return FL_OK;
    // (sigma_mode 2: every eligible band takes its split of fewest grid points)
    const double cands[4] = {2.0, 1.75, 1.5, 1.25};   // floors (1.25: only where the gain allows)
    double best_total = 0.0;
    std::vector<SplitChoice> best_ch;
    for (double smin : cands) {
        if (p.sigma_mode == 2 && smin != 1.25) continue;   // the lowest floor, fewest grid points
        const int mw = p.mw;   // sigma = 2; a split's own sigma may need more (best_split)
        std::vector<SplitChoice> ch;
        double total = 0.0;
        for (int b : nfft) {
            double c = 0.0;
            ch.push_back(best_split(p, p.bands[b], smin, mw, p.sigma_mode >= 2, &c));
            total += c;
        }
        if (best_ch.empty() || total < best_total) {
            best_total = total;
            best_ch = ch;
        }
    }
    bool any = false;
    double smin_used = 2.0;   // the smallest sigma actually chosen fixes m_w
    for (const SplitChoice& c : best_ch)
        if (c.P > 1) {
            any = true;
            smin_used = std::min(smin_used, ldexp(1.0, c.log2n) / (double)c.Nc);
        }
    if (!any) return FL_OK;
    p.mw = std::max(p.mw, window_width(p.eps_A, smin_used));
    p.sigma_min = smin_used;
    for (size_t i = 0; i < nfft.size(); ++i) {
        const SplitChoice c = best_ch[i];
        if (c.P == 1) continue;
        const int b = nfft[i];
        const int shift = p.bands[b].dev.log2n - c.log2n;   // node cells at the sub-band grid
        const int64_t n = (int64_t)1 << c.log2n;
        const double kb = M_PI * (2.0 - (double)c.Nc / (double)n);
        const int sub0 = (int)p.bands.size();
        for (int s = 0; s < c.P; ++s) {
            BandHost ch = p.bands[b];
            const int64_t k0 = s * c.Kp;
            ch.dev.parent = b;
            ch.dev.nsub = 0;
            ch.dev.k0 = k0;
            ch.dev.K = std::min<int64_t>(c.Kp, p.bands[b].dev.K - k0);
            ch.dev.Nm = c.Nc;
            ch.dev.n = n;
            ch.dev.log2n = c.log2n;
            ch.dev.kb = kb;
            ch.dev.c_off = p.bands[b].dev.c_off + k0;
            p.bands.push_back(ch);
        }
        BandDev& d = p.bands[b].dev;
        d.nsub = c.P;
        d.sub0 = sub0;
        d.n = n;
        d.log2n = c.log2n;
        d.kb = kb;
        cudaError_t e = launch_cell_shift(p.d_cell, p.bands[b].node_off, p.bands[b].nodes, shift, st);
        if (e != cudaSuccess) return cuda_fail(e, "fl_plan: sub-band cells");
    }
    return FL_OK;
}

// Plans the transforms Ns[i] x Ms[i], i < B, whose nodes are consecutive in
// `nodes` (a single plan is B = 1).  Every band of every transform gets an
// entry of one global band table, and each kernel launch of fl_execute covers
// all transforms at once.
static fl_status plan_multi(Plan& p, int B, const int64_t* Ns, const int64_t* Ms,
                            const double* nodes, int q, bool shared, cudaStream_t st) {
    fl_status s = select_common(p, q);
    if (s != FL_OK) return s;
    p.bands.clear();
    p.inst.assign(B, Instance());
    int64_t noff = 0, moff = 0, maxM = 0;
    for (int i = 0; i < B; ++i) {
        Instance& in = p.inst[i];
        in.N = Ns[i];
        in.M = Ms[i];
        in.noff = noff;
        in.moff = moff;
        in.src_off = shared ? 0 : moff;
        // a shared node set: the first transform of the same N is sorted, the
        // others copy its order (same bands, cells and routes)
        for (int j = 0; shared && j < i && in.twin < 0; ++j)
            if (Ns[j] == in.N) in.twin = j;
        noff += in.N;
        moff += in.M;
        maxM = std::max(maxM, in.M);
        if ((s = select_bands(p, in, i)) != FL_OK) return s;
    }
    p.N = noff;
    p.M = moff;
    p.levels = p.inst[0].levels;
    p.xi1 = p.inst[0].xi1;
    int nb = (int)p.bands.size();
    FL_CUDA(cudaMalloc((void**)&p.d_bands, nb * sizeof(BandDev)), "cudaMalloc bands");
    std::vector<BandDev> hb(nb);
    for (int b = 0; b < nb; ++b) hb[b] = p.bands[b].dev;
    FL_CUDA(cudaMemcpyAsync(p.d_bands, hb.data(), nb * sizeof(BandDev), cudaMemcpyHostToDevice, st),
            "copy bands");
    FL_CUDA(cudaMalloc((void**)&p.d_cheb, 2 * kMaxQ * sizeof(double)), "cudaMalloc cheb");
    FL_CUDA(cudaMalloc((void**)&p.d_cheb32, 4 * kMaxQ * sizeof(float)), "cudaMalloc cheb32");
    FL_CUDA(cudaMalloc(&p.d_z0, 2 * sizeof(double)), "cudaMalloc z0");

    // classify and sort the nodes of every transform into its slice
    const int64_t M = p.M;
    std::vector<int64_t> counts(nb, 0);
    if (M > 0) {
        FL_CUDA(cudaMalloc((void**)&p.d_ws, M * sizeof(double2)), "cudaMalloc nodes");
        FL_CUDA(cudaMalloc((void**)&p.d_perm, M * sizeof(int32_t)), "cudaMalloc perm");
        FL_CUDA(cudaMalloc((void**)&p.d_bandid, M * sizeof(int32_t)), "cudaMalloc band ids");
        FL_CUDA(cudaMalloc((void**)&p.d_cell, M * sizeof(int32_t)), "cudaMalloc cells");
        uint32_t *keys = nullptr, *keys2 = nullptr, *hist = nullptr;
        int32_t *vals = nullptr, *vals2 = nullptr;
        int64_t* dcount = nullptr;
        int* dflag = nullptr;
        const int64_t nblk = (maxM + 2047) / 2048;
        cudaError_t e = cudaSuccess;
        auto cleanup = [&]() {
            cudaFree(keys); cudaFree(keys2); cudaFree(hist); cudaFree(vals); cudaFree(vals2);
            cudaFree(dcount); cudaFree(dflag);
        };
        if ((e = cudaMalloc((void**)&keys, maxM * 4)) == cudaSuccess &&
            (e = cudaMalloc((void**)&keys2, maxM * 4)) == cudaSuccess &&
            (e = cudaMalloc((void**)&vals, maxM * 4)) == cudaSuccess &&
            (e = cudaMalloc((void**)&vals2, maxM * 4)) == cudaSuccess &&
            (e = cudaMalloc((void**)&hist, 256 * nblk * 4)) == cudaSuccess &&
            (e = cudaMalloc((void**)&dcount, nb * sizeof(int64_t))) == cudaSuccess &&
            (e = cudaMalloc((void**)&dflag, sizeof(int))) == cudaSuccess &&
            (e = cudaMemsetAsync(dcount, 0, nb * sizeof(int64_t), st)) == cudaSuccess &&
            (e = cudaMemsetAsync(dflag, 0, sizeof(int), st)) == cudaSuccess) {
            for (int i = 0; i < B && e == cudaSuccess; ++i) {
                const Instance& in = p.inst[i];
                if (in.twin >= 0) {
                    e = launch_copy_sorted(p, in, p.inst[in.twin], st);
                    continue;
                }
                if ((e = launch_classify(p, in, nodes, keys, vals, dcount, dflag, st)) == cudaSuccess &&
                    (e = radix_sort_pairs(keys, vals, keys2, vals2, hist, in.M, 32, st)) == cudaSuccess)
                    e = launch_permute(p, in, nodes, keys, vals, st);
            }
            int flag = 0;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(counts.data(), dcount, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess && flag) {
                cleanup();
                return fail(FL_EINVAL, p.xi_mode ? "fl_plan_xi: a node has Im w < 0, a non-finite part or |Re w| > 1/2"
                                                 : "fl_plan: a node has Im w < 0 or a non-finite part");
            }
        }
        cleanup();
        if (e != cudaSuccess) return cuda_fail(e, "fl_plan: node classification");
        for (const Instance& in : p.inst)
            if (in.twin >= 0)
                for (int lb = 0; lb <= in.levels; ++lb)
                    counts[in.band_base + lb] = counts[p.inst[in.twin].band_base + lb];
    }

    // routes, offsets and work lists
    p.grid_elems = p.D_elems = p.Y_elems = 0;
    p.xqc = p.xi_mode ? xi_chunk(p.q) : 0;
    p.small_work.clear();
    p.large_bands.clear();
    p.direct_work.clear();
    p.direct_ranges.clear();
    p.dadj_work32.clear();
    p.dadj_work64.clear();
    p.direct_nodes = p.direct_terms = p.dpart_elems = 0;
    p.n_direct_small = 0;
    p.n_dadj_small = 0;
    p.z0_nodes = 0;
    std::vector<DirectItem> small_items;
    std::vector<DirectAdjItem> small_adj;
    std::vector<int> nfft_bands;   // bands evaluated by an NFFT, in order
    for (int i = 0; i < B; ++i) {
        Instance& in = p.inst[i];
        in.z0_nodes = counts[in.band_base];
        p.z0_nodes += in.z0_nodes;
        int64_t off = in.moff + in.z0_nodes;
        p.bands[in.band_base].node_off = in.moff;
        p.bands[in.band_base].dev.node_off = in.moff;
        p.bands[in.band_base].nodes = in.z0_nodes;
        for (int lb = 1; lb <= in.levels; ++lb) {
            const int b = in.band_base + lb;
            BandHost& bh = p.bands[b];
            bh.nodes = counts[b];
            bh.node_off = off;
            off += counts[b];
            BandDev& d = bh.dev;
            d.node_off = bh.node_off;
            d.nodes = bh.nodes;
            d.route = bh.nodes > 0 ? route_of(p, bh) : 0;
            if (d.route == 2) {
                d.nchunk = (int)((d.K + kDirChunk - 1) / kDirChunk);
                d.dslot = p.dpart_elems;
                p.dpart_elems += bh.nodes * d.nchunk;
                p.direct_ranges.push_back({b, 0, bh.nodes, p.direct_nodes});
                p.direct_nodes += bh.nodes;
                p.direct_terms += bh.nodes * d.K;
                if (d.K <= kDirSmallK && bh.nodes >= kDirSmallMinNodes && p.prec == FL_FP32) {
                    for (int64_t n0 = 0; n0 < bh.nodes; n0 += kDirSmallNodes)
                        small_items.push_back({b, 0, bh.node_off + n0,
                                               (int)std::min<int64_t>(kDirSmallNodes, bh.nodes - n0), 0});
                } else {
                    for (int64_t n0 = 0; n0 < bh.nodes; n0 += kDirNodes)
                        for (int ch = 0; ch < d.nchunk; ++ch)
                            p.direct_work.push_back({b, ch, bh.node_off + n0,
                                                     (int)std::min<int64_t>(kDirNodes, bh.nodes - n0), 0});
                }
                if (!p.batched && d.K <= kDirSmallK) {
                    for (int64_t n0 = 0; n0 < bh.nodes; n0 += kDirAdjNodes)
                        small_adj.push_back({b, 0, bh.node_off + n0,
                                             (int)std::min<int64_t>(kDirAdjNodes, bh.nodes - n0), 0});
                } else if (!p.batched) {
                    for (int kl : {32, 16}) {
                        std::vector<DirectAdjItem>& v = kl == 32 ? p.dadj_work32 : p.dadj_work64;
                        const int64_t kc = (d.K + 32 * kl - 1) / (32 * kl);
                        for (int64_t n0 = 0; n0 < bh.nodes; n0 += kDirAdjNodes)
                            for (int64_t ch = 0; ch < kc; ++ch)
                                v.push_back({b, (int)ch, bh.node_off + n0,
                                             (int)std::min<int64_t>(kDirAdjNodes, bh.nodes - n0), 0});
                    }
                }
                continue;
            }
            if (d.route == 1) nfft_bands.push_back(b);
        }
    }
    // oversampling from the tolerance: split sparse bands into sub-bands
    if ((s = plan_splits(p, nfft_bands, st)) != FL_OK) return s;
    // a transform that copies its twin's nodes shares its twin's weight tables
    // (same N, bands and splits); shares_D[i] records that every band did
    std::vector<char> shares_D(B, 0);
    for (int i = 0; i < B; ++i) shares_D[i] = p.inst[i].twin >= 0 && !p.xi_mode;
    for (int b : nfft_bands) {
        const int nsub = p.bands[b].dev.nsub;
        const Instance& in = p.inst[p.bands[b].inst];
        const int tb = in.twin >= 0 ? b - in.band_base + p.inst[in.twin].band_base : -1;
        const bool twin_ok = tb >= 0 && p.bands[tb].dev.route == 1 && p.bands[tb].dev.nsub == nsub &&
                             p.bands[tb].dev.K == p.bands[b].dev.K;
        if (tb >= 0 && !twin_ok) shares_D[p.bands[b].inst] = 0;
        for (int c = 0; c < std::max(1, nsub); ++c) {
            const int g = nsub > 0 ? p.bands[b].dev.sub0 + c : b;
            BandDev& d = p.bands[g].dev;
            d.grid_off = p.grid_elems;
            p.grid_elems += (int64_t)d.nrhs * d.n;
            if (twin_ok && !p.xi_mode) {
                d.D_off = p.bands[nsub > 0 ? p.bands[tb].dev.sub0 + c : tb].dev.D_off;
            } else if (p.xi_mode) {
                // exponent-major rows of whole spreading chunks, 16-byte aligned
                d.dld = d.nrhs == 1 ? 1 : (d.nrhs + p.xqc - 1) / p.xqc * p.xqc;
                p.D_elems = (p.D_elems + 3) & ~(int64_t)3;
                d.D_off = p.D_elems;
                p.D_elems += (int64_t)d.dld * d.K;
            } else {
                d.D_off = p.D_elems;
                p.D_elems += (int64_t)d.nrhs * d.K;
            }
            if (d.log2n <= kSmallMaxLog2) {
                // 4096 points per CTA (256 threads x 16); n = 32 at 8 points per thread
                const int per = std::max(1, (int)((d.log2n >= 6 ? 4096 : 2048) / d.n));
                for (int s0 = 0; s0 < d.nrhs; s0 += per)
                    p.small_work.push_back({g, s0, std::min(per, d.nrhs - s0), d.log2n});
            } else {
                p.large_bands.push_back(g);
            }
        }
    }
    // few direct items (a handful of sparse bands): half as many nodes per
    // item, so the launch still covers the GPU several times over
    if (!p.direct_work.empty() && (int64_t)p.direct_work.size() < kDirFewItems) {
        std::vector<DirectItem> halves;
        for (const DirectItem& it : p.direct_work) {
            const int h = std::min(it.nnodes, kDirNodes / 2);
            halves.push_back({it.band, it.chunk, it.node0, h, 0});
            if (it.nnodes > h) halves.push_back({it.band, it.chunk, it.node0 + h, it.nnodes - h, 0});
        }
        p.direct_work.swap(halves);
    }
    p.n_direct_small = (int64_t)small_items.size();
    p.direct_work.insert(p.direct_work.end(), small_items.begin(), small_items.end());
    p.n_dadj_small = (int64_t)small_adj.size();
    p.dadj_work32.insert(p.dadj_work32.end(), small_adj.begin(), small_adj.end());
    p.dadj_work64.insert(p.dadj_work64.end(), small_adj.begin(), small_adj.end());
    build_pass_groups(p);
    if ((s = build_fused(p, st)) != FL_OK) return s;
    if ((int)p.bands.size() != nb) {   // sub-bands were appended: a larger table
        FL_CUDA(cudaStreamSynchronize(st), "fl_plan: synchronise");
        FL_CUDA(cudaFree(p.d_bands), "cudaFree bands");
        p.d_bands = nullptr;
        nb = (int)p.bands.size();
        hb.resize(nb);
        FL_CUDA(cudaMalloc((void**)&p.d_bands, nb * sizeof(BandDev)), "cudaMalloc bands");
    }
    for (int b = 0; b < nb; ++b) hb[b] = p.bands[b].dev;
    FL_CUDA(cudaMemcpyAsync(p.d_bands, hb.data(), nb * sizeof(BandDev), cudaMemcpyHostToDevice, st),
            "copy bands");
    if (p.prec == FL_FP32 && !p.xi_mode && p.M > 0) {
        FL_CUDA(cudaMalloc((void**)&p.d_ntab, p.M * sizeof(uint4)), "cudaMalloc node records");
        FL_CUDA(build_node_table(p, st), "fl_plan: node records");
    }
    // complex128 I/O for FP64 and float pairs; real tables double or float pairs
    const size_t cs = p.prec != FL_FP32 ? 16 : 8, rs = cs / 2;
    if (!p.small_work.empty()) {
        FL_CUDA(cudaMalloc((void**)&p.d_small, p.small_work.size() * sizeof(SmallWork)), "cudaMalloc work");
        FL_CUDA(cudaMemcpyAsync(p.d_small, p.small_work.data(), p.small_work.size() * sizeof(SmallWork),
                                cudaMemcpyHostToDevice, st),
                "copy work");
    }
    if (!p.pass_items.empty()) {
        FL_CUDA(cudaMalloc((void**)&p.d_pass, p.pass_items.size() * sizeof(PassItem)), "cudaMalloc pass items");
        FL_CUDA(cudaMemcpyAsync(p.d_pass, p.pass_items.data(), p.pass_items.size() * sizeof(PassItem),
                                cudaMemcpyHostToDevice, st),
                "copy pass items");
    }
    if (!p.direct_work.empty()) {
        FL_CUDA(cudaMalloc((void**)&p.d_direct, p.direct_work.size() * sizeof(DirectItem)),
                "cudaMalloc direct work");
        FL_CUDA(cudaMemcpyAsync(p.d_direct, p.direct_work.data(),
                                p.direct_work.size() * sizeof(DirectItem), cudaMemcpyHostToDevice, st),
                "copy direct work");
        FL_CUDA(cudaMalloc((void**)&p.d_dranges, p.direct_ranges.size() * sizeof(DirectRange)),
                "cudaMalloc direct ranges");
        FL_CUDA(cudaMemcpyAsync(p.d_dranges, p.direct_ranges.data(),
                                p.direct_ranges.size() * sizeof(DirectRange), cudaMemcpyHostToDevice, st),
                "copy direct ranges");
        FL_CUDA(cudaMalloc(&p.d_dpart, p.dpart_elems * cs), "cudaMalloc direct partials");
        std::vector<DirectAdjItem>& adj = p.prec != FL_FP32 ? p.dadj_work64 : p.dadj_work32;
        DirectAdjItem*& d_adj = p.prec != FL_FP32 ? p.d_dadj64 : p.d_dadj32;
        if (!adj.empty()) {
            FL_CUDA(cudaMalloc((void**)&d_adj, adj.size() * sizeof(DirectAdjItem)), "cudaMalloc adjoint work");
            FL_CUDA(cudaMemcpyAsync(d_adj, adj.data(), adj.size() * sizeof(DirectAdjItem),
                                    cudaMemcpyHostToDevice, st),
                    "copy adjoint work");
        }
        FL_CUDA(cudaMalloc(&p.d_cdir, p.N * cs), "cudaMalloc direct adjoint");
    }
    // adjoint of the NFFT bands (single plans): per-node taps and weights, cell list
    p.cell_bands.clear();
    p.cells_total = p.cells_dense = 0;
    p.n_sparse_cb = 0;
    if (!p.batched && M > 0) {
        // dense: on average >= 32 window contributions per cell (warp per cell)
        auto dense = [&](const BandHost& bh) { return bh.nodes * 2 * p.mw >= 32 * bh.dev.n; };
        for (int b = 0; b < nb; ++b) {
            const BandDev& d = p.bands[b].dev;
            if (d.route != 1 || d.nsub > 0 || dense(p.bands[b])) continue;
            p.cell_bands.push_back({b, 0, p.cells_total});
            p.cells_total += d.n;
        }
        p.n_sparse_cb = (int)p.cell_bands.size();
        for (int b = 0; b < nb; ++b) {
            const BandDev& d = p.bands[b].dev;
            if (d.route != 1 || d.nsub > 0 || !dense(p.bands[b])) continue;
            p.cell_bands.push_back({b, 0, p.cells_dense});
            p.cells_dense += d.n;
        }
        if (!p.cell_bands.empty()) {
            FL_CUDA(cudaMalloc((void**)&p.d_cell_bands, p.cell_bands.size() * sizeof(Plan::CellBand)),
                    "cudaMalloc cell bands");
            FL_CUDA(cudaMemcpyAsync(p.d_cell_bands, p.cell_bands.data(),
                                    p.cell_bands.size() * sizeof(Plan::CellBand), cudaMemcpyHostToDevice, st),
                    "copy cell bands");
            FL_CUDA(cudaMalloc(&p.d_sp_phi, (size_t)M * 2 * p.mw * rs), "cudaMalloc adjoint taps");
            FL_CUDA(cudaMalloc(&p.d_sp_L, (size_t)M * p.q * rs), "cudaMalloc adjoint weights");
            FL_CUDA(cudaMalloc(&p.d_sp_rv, (size_t)M * cs), "cudaMalloc adjoint residuals");
        }
    }
    if (p.grid_elems) FL_CUDA(cudaMalloc(&p.d_grid, p.grid_elems * cs), "cudaMalloc grids");
    if (p.D_elems) FL_CUDA(cudaMalloc(&p.d_D, p.D_elems * rs), "cudaMalloc weights");
    if (p.D_elems && p.xi_mode)   // the padding of the exponent-major rows
        FL_CUDA(cudaMemsetAsync(p.d_D, 0, p.D_elems * rs, st), "clear weights");
    if (p.Y_elems) FL_CUDA(cudaMalloc(&p.d_Y, p.Y_elems * cs), "cudaMalloc intermediate");
    if (p.Y_elems || !p.small_work.empty()) {   // stage twiddles of the passes and the small FFTs
        FL_CUDA(cudaMalloc(&p.d_tw, (size_t)(kTwEntries + (p.prec == FL_FP64_FF ? 8192 : 0)) * cs),
                "cudaMalloc twiddles");
        FL_CUDA(build_twiddles(p, st), "fl_plan: twiddles");
    }
    if (p.prec == FL_FP64_FF)
        FL_CUDA(cudaMalloc(&p.d_cff, (size_t)p.N * sizeof(ffc)), "cudaMalloc float-pair coefficients");
    FL_CUDA(build_cheb(p, st), "fl_plan: tables");
    for (int i = 0; i < B; ++i)
        if (!shares_D[i]) FL_CUDA(build_tables(p, p.inst[i], st), "fl_plan: tables");
    FL_CUDA(cudaStreamSynchronize(st), "fl_plan: synchronise");
    p.scratch_bytes = (double)p.grid_elems * cs + (double)p.D_elems * rs + (double)p.Y_elems * cs +
                      (double)M * (sizeof(double2) + 8) + (double)p.dpart_elems * cs +
                      (p.direct_work.empty() ? 0.0 : (double)p.N * cs);
    // algorithmic bytes of one execute: c once, D once, each grid written and read
    // once per FFT pass, the nodes, and f
    double mb = (double)p.N * cs + (double)p.D_elems * rs + (double)M * (sizeof(double2) + 8 + cs);
    for (int b = 0; b < nb; ++b) {
        const BandDev& d = p.bands[b].dev;
        if (d.route != 1 || d.nsub > 0) continue;   // split bands: their sub-bands
        const double g = (double)d.nrhs * d.n * cs;
        if (d.fused) {   // Y write + read; entries read, partials written and gathered
            const int NQ = (pass_tiles(8, (d.log2n + 1) / 2, FL_P2_THREADS_F32) + 3) / 4;
            mb += 2.0 * g + (double)d.nrhs * p.bands[b].fentries * (8.0 + 16.0 * NQ + 8.0) +
                  (double)d.nrhs * p.bands[b].nodes * d.pparts * cs;
            continue;
        }
        mb += (d.log2n <= kSmallMaxLog2) ? g : 3.0 * g;   // small: write; large: Y write+read, grid write
        mb += std::min<double>(g, (double)p.bands[b].nodes * d.nrhs * 2 * p.mw * cs);   // gather
    }
    if (!p.direct_work.empty()) mb += (double)p.direct_work.size() * kDirChunk * cs;   // c tiles
    p.model_bytes = mb;
    return FL_OK;
}


// Everything that defines a Fourier-Laplace plan besides the route bias.
struct PlanSpec {
    int B;
    const int64_t* Ns;
    const int64_t* Ms;
    const double* nodes;
    int q;
    double eps;
    fl_precision prec;
    bool batched;
    int route_mode;
    int rhs_per_launch;
    bool use_graph;
    int variant;
    int fuse_mode;
    int sigma_mode;
    bool shared_nodes;
};

static fl_status build_plan(const PlanSpec& sp, double bias, fl_plan_s** out, cudaStream_t st) {
    fl_plan_s* h = new (std::nothrow) fl_plan_s();
    if (!h) return fail(FL_ENOMEM, "fl_plan: host allocation");
    h->p.kind = 0;
    h->p.batched = sp.batched;
    h->p.prec = sp.prec;
    h->p.eps = sp.eps;
    h->p.route_mode = sp.route_mode;
    h->p.direct_bias = bias;
    h->p.rhs_per_launch = sp.rhs_per_launch;
    h->p.use_graph = sp.use_graph;
    h->p.variant = sp.variant;
    h->p.fuse_mode = sp.fuse_mode;
    h->p.sigma_mode = sp.sigma_mode;
    fl_status s = plan_multi(h->p, sp.B, sp.Ns, sp.Ms, sp.nodes, sp.q, sp.shared_nodes, st);
    if (s != FL_OK) {
        delete h;
        return s;
    }
    *out = h;
    return FL_OK;
}

// Autotuner: plans the workload for candidate settings, times three executes
// of each (CUDA events on the caller's stream, after one warm-up, on zero
// coefficients: the work does not depend on the values), and keeps the
// fastest.  Coordinate search, each setting from the best so far: the route
// bias (route 0), then -- where the caller left them at their defaults -- the
// oversampling (sigma from the tolerance or 2), the fused gather (by cost or
// never) and the grids per four-step launch.  The choice is cached for the
// process by a signature of the workload (sizes, eps, precision, the caller's
// settings and the node count of every band), so planning the same workload
// again costs one plan.
struct Tuned {
    double bias;
    int sigma_mode, fuse_mode, rhs;
};
static std::vector<std::pair<uint64_t, Tuned>> g_tuned;
static std::mutex g_tuned_mutex;

static uint64_t plan_signature(const Plan& p, const PlanSpec& sp) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    mix((uint64_t)p.N);
    mix((uint64_t)p.M);
    mix((uint64_t)p.inst.size());
    mix((uint64_t)p.prec);
    uint64_t e;
    memcpy(&e, &p.eps, sizeof(e));
    mix(e);
    mix((uint64_t)p.q);
    mix((uint64_t)p.variant);
    mix((uint64_t)sp.route_mode);
    mix((uint64_t)sp.sigma_mode);
    mix((uint64_t)sp.fuse_mode);
    mix((uint64_t)sp.rhs_per_launch);
    for (const Instance& in : p.inst) mix((uint64_t)(in.twin + 1));
    for (const BandHost& bh : p.bands) mix((uint64_t)bh.nodes * 131 + (uint64_t)bh.local);
    return h;
}

static fl_status time_plan(Plan& p, cudaStream_t st, double* ms) {
    const size_t cs = p.prec != FL_FP32 ? 16 : 8;
    void *c = nullptr, *f = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&c, std::max<int64_t>(1, p.N) * cs);
    if (e == cudaSuccess) e = cudaMalloc(&f, std::max<int64_t>(1, p.M) * cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(c, 0, std::max<int64_t>(1, p.N) * cs, st);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int64_t launches = p.launches;
    if (e == cudaSuccess) e = run_forward(p, c, f, false, st);
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = run_forward(p, c, f, false, st);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    p.launches = launches;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(c);
    cudaFree(f);
    if (e != cudaSuccess) return cuda_fail(e, "fl_plan: autotune");
    *ms = t / 3.0;
    return FL_OK;
}

static PlanSpec with_tuned(const PlanSpec& sp, const Tuned& t) {
    PlanSpec r = sp;
    r.sigma_mode = t.sigma_mode;
    r.fuse_mode = t.fuse_mode;
    r.rhs_per_launch = t.rhs;
    return r;
}

static void set_tuned(Plan& p, const Tuned& t) {
    p.tuned_bias = t.bias;
    p.tuned_sigma_mode = t.sigma_mode;
    p.tuned_fuse_mode = t.fuse_mode;
    p.tuned_rhs = t.rhs;
}

static fl_status build_plan_tuned(const PlanSpec& sp, double bias, bool autotune, fl_plan_s** out,
                                  cudaStream_t st) {
    fl_plan_s* h = nullptr;
    fl_status s = build_plan(sp, bias, &h, st);
    if (s != FL_OK || !autotune) {
        *out = h;
        return s;
    }
    const uint64_t sig = plan_signature(h->p, sp);
    const Tuned start{bias, sp.sigma_mode, sp.fuse_mode, sp.rhs_per_launch};
    bool hit = false;
    Tuned cached = start;
    {
        std::lock_guard<std::mutex> lock(g_tuned_mutex);
        for (const auto& kv : g_tuned)
            if (kv.first == sig) {
                cached = kv.second;
                hit = true;
            }
    }
    if (hit) {
        if (cached.bias != start.bias || cached.sigma_mode != start.sigma_mode ||
            cached.fuse_mode != start.fuse_mode || cached.rhs != start.rhs) {
            delete h;
            h = nullptr;
            if ((s = build_plan(with_tuned(sp, cached), cached.bias, &h, st)) != FL_OK) return s;
        }
        set_tuned(h->p, cached);
        *out = h;
        return FL_OK;
    }
    double best_ms = 0;
    if ((s = time_plan(h->p, st, &best_ms)) != FL_OK) {
        delete h;
        return s;
    }
    Tuned best = start;
    auto try_cand = [&](const Tuned& t) -> fl_status {
        fl_plan_s* c = nullptr;
        fl_status r = build_plan(with_tuned(sp, t), t.bias, &c, st);
        if (r != FL_OK) return r;
        double ms = 0;
        if ((r = time_plan(c->p, st, &ms)) != FL_OK) {
            delete c;
            return r;
        }
        if (ms < best_ms) {
            delete h;
            h = c;
            best_ms = ms;
            best = t;
        } else {
            delete c;
        }
        return FL_OK;
    };
    std::vector<Tuned> cands;
    const bool fp32 = sp.prec == FL_FP32;
    if (sp.route_mode == 0)
        for (double cand : {0.125, 0.25, 0.5, 2.0, 4.0, 8.0}) {
            Tuned t = best;
            t.bias = cand;
            if ((s = try_cand(t)) != FL_OK) break;
        }
    if (s == FL_OK && fp32 && sp.sigma_mode == 0) {
        Tuned t = best;
        t.sigma_mode = 1;
        s = try_cand(t);
    }
    if (s == FL_OK && fp32 && sp.fuse_mode == 0) {
        Tuned t = best;
        t.fuse_mode = 1;
        s = try_cand(t);
    }
    if (s == FL_OK && sp.rhs_per_launch == 0)
        for (int r : {12, 36}) {
            Tuned t = best;
            t.rhs = r;
            if ((s = try_cand(t)) != FL_OK) break;
        }
    if (s != FL_OK) {
        delete h;
        return s;
    }
    {
        std::lock_guard<std::mutex> lock(g_tuned_mutex);
        g_tuned.push_back({sig, best});
    }
    set_tuned(h->p, best);
    *out = h;
    return FL_OK;
}

// fl_execute through a CUDA graph of its launches, captured on the first call
// (and again when the buffers or the stream change), then replayed.
static cudaError_t forward_graphed(Plan& p, const void* c, void* f, cudaStream_t st) {
    if (!p.use_graph || p.timing || st == nullptr) return run_forward(p, c, f, false, st);
    if (!p.gexec || p.g_c != c || p.g_f != f || p.g_st != st) {
        if (p.gexec) {
            cudaGraphExecDestroy(p.gexec);
            p.gexec = nullptr;
        }
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const int64_t launches = p.launches;
        cudaError_t er = run_forward(p, c, f, false, st);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (er != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return er;
        }
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&p.gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            p.gexec = nullptr;
            return e;
        }
        p.graph_launches = p.launches - launches;
        p.launches = launches;
        p.g_c = c;
        p.g_f = f;
        p.g_st = st;
    }
    p.launches += p.graph_launches;
    return cudaGraphLaunch(p.gexec, st);
}

// Batched plans with per-transform buffers: element e of the concatenation
// belongs to transform b with off[b] <= e < off[b + 1] (binary search);
// pack copies the callers' arrays into the concatenation, unpack back out.
template <typename E>
__global__ void k_batch_pack(int B, const int64_t* __restrict__ off, const E* const* __restrict__ src,
                             int64_t total, E* __restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int lo = 0, hi = B;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= e) lo = mid;
        else hi = mid;
    }
    dst[e] = src[lo][e - off[lo]];
}

template <typename E>
__global__ void k_batch_unpack(int B, const int64_t* __restrict__ off, const E* __restrict__ src,
                               int64_t total, E* const* __restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int lo = 0, hi = B;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= e) lo = mid;
        else hi = mid;
    }
    dst[lo][e - off[lo]] = src[e];
}

// pack: c pointers -> d_stage_c; else d_stage_f -> f pointers (offsets and
// pointers from d_boff / d_bptr).
static cudaError_t launch_batch_pack(Plan& p, size_t cs, bool pack, cudaStream_t st) {
    const int B = (int)p.inst.size();
    const int64_t total = pack ? p.N : p.M;
    if (total == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((total + 255) / 256);
    const int64_t* off = pack ? p.d_boff : p.d_boff + B + 1;
    if (cs == 16) {
        if (pack)
            k_batch_pack<double2><<<grid, 256, 0, st>>>(B, off, (const double2* const*)p.d_bptr, total,
                                                        (double2*)p.d_stage_c);
        else
            k_batch_unpack<double2><<<grid, 256, 0, st>>>(B, off, (const double2*)p.d_stage_f, total,
                                                          (double2* const*)(p.d_bptr + B));
    } else {
        if (pack)
            k_batch_pack<float2><<<grid, 256, 0, st>>>(B, off, (const float2* const*)p.d_bptr, total,
                                                       (float2*)p.d_stage_c);
        else
            k_batch_unpack<float2><<<grid, 256, 0, st>>>(B, off, (const float2*)p.d_stage_f, total,
                                                         (float2* const*)(p.d_bptr + B));
    }
    ++p.launches;
    return cudaGetLastError();
}

}  // namespace fl

using namespace fl;

extern "C" {

const char* fl_last_error(void) { return g_err.c_str(); }

const char* fl_version(void) { return "fastfl 0.1 (sm_103a)"; }

static bool options_valid(const fl_options* opt) {
    return !opt || (opt->route >= 0 && opt->route <= 2 && opt->direct_bias >= 0.0 &&
                    opt->rhs_per_launch >= 0 && opt->variant >= 0 && opt->variant <= 1 &&
                    opt->fuse_gather >= 0 && opt->fuse_gather <= 2 && opt->oversampling >= 0 &&
                    opt->oversampling <= 2 && opt->shared_nodes >= 0 && opt->shared_nodes <= 1);
}

fl_status fl_plan(fl_plan_t* out, int64_t N, int64_t M, const double* nodes_dev, int q, double eps,
                  fl_precision prec, void* stream) {
    return fl_plan_ex(out, N, M, nodes_dev, q, eps, prec, nullptr, stream);
}

fl_status fl_plan_ex(fl_plan_t* out, int64_t N, int64_t M, const double* nodes_dev, int q,
                     double eps, fl_precision prec, const fl_options* opt, void* stream) {
    g_err.clear();
    if (!options_valid(opt))
        return fail(FL_EINVAL, "fl_plan: invalid options");
    if (!out) return fail(FL_EINVAL, "fl_plan: out is NULL");
    *out = nullptr;
    if (N < 1 || M < 0) return fail(FL_EINVAL, "fl_plan: need N >= 1 and M >= 0");
    if (N > ((int64_t)1 << 23)) return fail(FL_EUNSUPPORTED, "fl_plan: N above 2^23");
    if (M > ((int64_t)1 << 31) - 1) return fail(FL_EUNSUPPORTED, "fl_plan: M above 2^31 - 1");
    if (!(eps > 0.0 && eps < 1.0)) return fail(FL_EINVAL, "fl_plan: eps must lie in (0, 1)");
    if (q < 0 || q > kMaxQ) return fail(FL_EINVAL, "fl_plan: q must lie in [0, 40]");
    if (prec != FL_FP32 && prec != FL_FP64 && prec != FL_FP64_FF)
        return fail(FL_EINVAL, "fl_plan: unknown precision");
    if (M > 0 && !nodes_dev) return fail(FL_EINVAL, "fl_plan: nodes is NULL");
    PlanSpec sp{1, &N, &M, nodes_dev, q, eps, prec, false,
                 opt ? opt->route : 0, opt ? opt->rhs_per_launch : 0, opt ? opt->use_graph != 0 : false,
                 opt ? opt->variant : 0, opt ? opt->fuse_gather : 0, opt ? opt->oversampling : 0,
                 false};
    const double bias = (opt && opt->direct_bias > 0.0) ? opt->direct_bias : 1.0;
    fl_plan_s* h = nullptr;
    fl_status s = build_plan_tuned(sp, bias, opt && opt->autotune, &h, (cudaStream_t)stream);
    if (s != FL_OK) return s;
    *out = h;
    return FL_OK;
}

fl_status fl_execute(fl_plan_t h, const void* c_dev, void* f_dev, void* stream) {
    if (!h || h->p.kind != 0) return fail(FL_EINVAL, "fl_execute: not a Fourier-Laplace plan");
    if (h->p.M > 0 && (!c_dev || !f_dev)) return fail(FL_EINVAL, "fl_execute: NULL buffer");
    if (h->p.batched) return fail(FL_EINVAL, "fl_execute: batched plan (use fl_execute_batched)");
    cudaError_t e = h->p.xi_mode ? run_forward_xi(h->p, c_dev, f_dev, (cudaStream_t)stream)
                                 : forward_graphed(h->p, c_dev, f_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fl_execute");
    return FL_OK;
}

fl_status fl_execute_deriv(fl_plan_t h, const void* c_dev, void* f_dev, void* stream) {
    if (!h || h->p.kind != 0) return fail(FL_EINVAL, "fl_execute_deriv: not a Fourier-Laplace plan");
    if (h->p.M > 0 && (!c_dev || !f_dev)) return fail(FL_EINVAL, "fl_execute_deriv: NULL buffer");
    if (h->p.batched) return fail(FL_EUNSUPPORTED, "fl_execute_deriv: batched plans are forward only");
    if (h->p.xi_mode) return fail(FL_EUNSUPPORTED, "fl_execute_deriv: real-exponent plans are forward only");
    cudaError_t e = run_forward(h->p, c_dev, f_dev, true, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fl_execute_deriv");
    return FL_OK;
}

fl_status fl_grad_w(fl_plan_t h, const void* c_dev, const void* r_dev, void* gw_dev, void* stream) {
    if (!h || h->p.kind != 0) return fail(FL_EINVAL, "fl_grad_w: not a Fourier-Laplace plan");
    if (h->p.M > 0 && (!c_dev || !r_dev || !gw_dev)) return fail(FL_EINVAL, "fl_grad_w: NULL buffer");
    if (h->p.batched) return fail(FL_EUNSUPPORTED, "fl_grad_w: batched plans are forward only");
    if (h->p.xi_mode) return fail(FL_EUNSUPPORTED, "fl_grad_w: real-exponent plans are forward only");
    cudaError_t e = run_forward(h->p, c_dev, gw_dev, true, (cudaStream_t)stream, r_dev);
    if (e != cudaSuccess) return cuda_fail(e, "fl_grad_w");
    return FL_OK;
}

fl_status fl_execute_host(fl_plan_t h, const void* c_host, void* f_host, void* stream) {
    if (!h || h->p.kind != 0) return fail(FL_EINVAL, "fl_execute_host: not a Fourier-Laplace plan");
    Plan& p = h->p;
    if (!c_host || (p.M > 0 && !f_host)) return fail(FL_EINVAL, "fl_execute_host: NULL buffer");
    const size_t cs = p.prec != FL_FP32 ? 16 : 8;
    cudaStream_t st = (cudaStream_t)stream;
    if (!p.d_stage_c) FL_CUDA(cudaMalloc(&p.d_stage_c, p.N * cs), "cudaMalloc staging");
    if (!p.d_stage_f && p.M > 0) FL_CUDA(cudaMalloc(&p.d_stage_f, p.M * cs), "cudaMalloc staging");
    FL_CUDA(cudaMemcpyAsync(p.d_stage_c, c_host, p.N * cs, cudaMemcpyHostToDevice, st), "copy c");
    FL_CUDA(p.xi_mode ? run_forward_xi(p, p.d_stage_c, p.d_stage_f, st)
                      : forward_graphed(p, p.d_stage_c, p.d_stage_f, st),
            "fl_execute_host");
    if (p.M > 0)
        FL_CUDA(cudaMemcpyAsync(f_host, p.d_stage_f, p.M * cs, cudaMemcpyDeviceToHost, st), "copy f");
    FL_CUDA(cudaStreamSynchronize(st), "fl_execute_host: synchronise");
    return FL_OK;
}

fl_status fl_adjoint(fl_plan_t h, const void* r_dev, void* c_out_dev, void* stream) {
    if (!h || h->p.kind != 0) return fail(FL_EINVAL, "fl_adjoint: not a Fourier-Laplace plan");
    if (!c_out_dev || (h->p.M > 0 && !r_dev)) return fail(FL_EINVAL, "fl_adjoint: NULL buffer");
    if (h->p.batched) return fail(FL_EUNSUPPORTED, "fl_adjoint: batched plans are forward only");
    cudaError_t e = run_adjoint(h->p, r_dev, c_out_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fl_adjoint");
    return FL_OK;
}

fl_status fl_transposed(fl_plan_t h, const void* g_dev, void* out_dev, void* stream) {
    if (!h || h->p.kind != 0) return fail(FL_EINVAL, "fl_transposed: not a Fourier-Laplace plan");
    if (!out_dev || (h->p.M > 0 && !g_dev)) return fail(FL_EINVAL, "fl_transposed: NULL buffer");
    if (h->p.batched) return fail(FL_EUNSUPPORTED, "fl_transposed: batched plans are forward only");
    cudaError_t e = run_transposed(h->p, g_dev, out_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fl_transposed");
    return FL_OK;
}

fl_status fl_plan_xi(fl_plan_t* out, int64_t N, const double* xi_dev, int64_t M,
                     const double* nodes_dev, int q, double eps, fl_precision prec, void* stream) {
    g_err.clear();
    if (!out) return fail(FL_EINVAL, "fl_plan_xi: out is NULL");
    *out = nullptr;
    if (N < 1 || M < 0) return fail(FL_EINVAL, "fl_plan_xi: need N >= 1 and M >= 0");
    if (N > ((int64_t)1 << 22) || M > ((int64_t)1 << 31) - 1)
        return fail(FL_EUNSUPPORTED, "fl_plan_xi: N above 2^22 or M above 2^31 - 1");
    if (!(eps > 0.0 && eps < 1.0)) return fail(FL_EINVAL, "fl_plan_xi: eps must lie in (0, 1)");
    if (q < 0 || q > kMaxQ) return fail(FL_EINVAL, "fl_plan_xi: q must lie in [0, 40]");
    if (prec != FL_FP32 && prec != FL_FP64) return fail(FL_EINVAL, "fl_plan_xi: unknown precision");
    if (!xi_dev || (M > 0 && !nodes_dev)) return fail(FL_EINVAL, "fl_plan_xi: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> xh(N);
    FL_CUDA(cudaMemcpyAsync(xh.data(), xi_dev, N * sizeof(double), cudaMemcpyDeviceToHost, st), "copy xi");
    FL_CUDA(cudaStreamSynchronize(st), "fl_plan_xi: synchronise");
    std::vector<std::pair<double, int32_t>> order(N);
    for (int64_t k = 0; k < N; ++k) {
        if (!(xh[k] >= 1.0) || !std::isfinite(xh[k]))
            return fail(FL_EINVAL, "fl_plan_xi: every exponent must be finite and >= 1");
        order[k] = {xh[k], (int32_t)k};
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<double, int32_t>& a, const std::pair<double, int32_t>& b) {
                         return a.first < b.first;
                     });
    fl_plan_s* h = new (std::nothrow) fl_plan_s();
    if (!h) return fail(FL_ENOMEM, "fl_plan_xi: host allocation");
    Plan& p = h->p;
    p.kind = 0;
    p.prec = prec;
    p.eps = eps;
    p.route_mode = 1;
    p.xi_mode = true;
    p.h_xis.resize(N);
    std::vector<int32_t> perm(N);
    for (int64_t k = 0; k < N; ++k) {
        p.h_xis[k] = order[k].first;
        perm[k] = order[k].second;
    }
    auto bail = [&](fl_status s) {
        delete h;
        return s;
    };
    cudaError_t e = cudaMalloc((void**)&p.d_xis, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p.d_xperm, N * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p.d_xis, p.h_xis.data(), N * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p.d_xperm, perm.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "fl_plan_xi: exponents"));
    fl_status s = plan_multi(p, 1, &N, &M, nodes_dev, q, false, st);
    if (s != FL_OK) return bail(s);
    e = build_xi_tables(p, st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "fl_plan_xi: tables"));
    *out = h;
    return FL_OK;
}

fl_status fl_plan_batched(fl_plan_t* out, int B, const int64_t* N_host, const int64_t* M_host,
                          const double* nodes_dev, int q, double eps, fl_precision prec,
                          const fl_options* opt, void* stream) {
    g_err.clear();
    if (!out) return fail(FL_EINVAL, "fl_plan_batched: out is NULL");
    *out = nullptr;
    if (B < 1 || !N_host || !M_host) return fail(FL_EINVAL, "fl_plan_batched: need B >= 1 and sizes");
    int64_t Mtot = 0, Ntot = 0;
    for (int i = 0; i < B; ++i) {
        if (N_host[i] < 1 || M_host[i] < 0)
            return fail(FL_EINVAL, "fl_plan_batched: need N_i >= 1 and M_i >= 0");
        if (N_host[i] > ((int64_t)1 << 23)) return fail(FL_EUNSUPPORTED, "fl_plan_batched: N_i above 2^23");
        Ntot += N_host[i];
        Mtot += M_host[i];
    }
    if (Mtot > ((int64_t)1 << 31) - 1 || Ntot > ((int64_t)1 << 40))
        return fail(FL_EUNSUPPORTED, "fl_plan_batched: sum of M_i above 2^31 - 1");
    if (!(eps > 0.0 && eps < 1.0)) return fail(FL_EINVAL, "fl_plan_batched: eps must lie in (0, 1)");
    if (q < 0 || q > kMaxQ) return fail(FL_EINVAL, "fl_plan_batched: q must lie in [0, 40]");
    if (prec != FL_FP32 && prec != FL_FP64 && prec != FL_FP64_FF)
        return fail(FL_EINVAL, "fl_plan_batched: unknown precision");
    if (Mtot > 0 && !nodes_dev) return fail(FL_EINVAL, "fl_plan_batched: nodes is NULL");
    if (!options_valid(opt))
        return fail(FL_EINVAL, "fl_plan_batched: invalid options");
    const bool shared = opt && opt->shared_nodes;
    for (int i = 1; shared && i < B; ++i)
        if (M_host[i] != M_host[0])
            return fail(FL_EINVAL, "fl_plan_batched: shared nodes need every M_i equal to M_0");
    PlanSpec sp{B, N_host, M_host, nodes_dev, q, eps, prec, true, opt ? opt->route : 0,
                 opt ? opt->rhs_per_launch : 0, opt ? opt->use_graph >= 0 : true,
                 opt ? opt->variant : 0, opt ? opt->fuse_gather : 0, opt ? opt->oversampling : 0,
                 shared};
    const double bias = (opt && opt->direct_bias > 0.0) ? opt->direct_bias : 1.0;
    fl_plan_s* h = nullptr;
    fl_status s = build_plan_tuned(sp, bias, opt && opt->autotune, &h, (cudaStream_t)stream);
    if (s != FL_OK) return s;
    *out = h;
    return FL_OK;
}

fl_status fl_execute_batched(fl_plan_t h, const void* c_dev, void* f_dev, void* stream) {
    if (!h || h->p.kind != 0 || !h->p.batched)
        return fail(FL_EINVAL, "fl_execute_batched: not a batched Fourier-Laplace plan");
    if (h->p.M > 0 && (!c_dev || !f_dev)) return fail(FL_EINVAL, "fl_execute_batched: NULL buffer");
    cudaError_t e = forward_graphed(h->p, c_dev, f_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fl_execute_batched");
    return FL_OK;
}

fl_status fl_plan_batched_ptrs(fl_plan_t* out, int B, const int64_t* N_host, const int64_t* M_host,
                               const double* const* nodes_host, int q, double eps, fl_precision prec,
                               const fl_options* opt, void* stream) {
    g_err.clear();
    if (!out) return fail(FL_EINVAL, "fl_plan_batched_ptrs: out is NULL");
    *out = nullptr;
    if (B < 1 || !N_host || !M_host) return fail(FL_EINVAL, "fl_plan_batched_ptrs: need B >= 1 and sizes");
    if (opt && opt->shared_nodes)   // one node set: the first pointer
        return fl_plan_batched(out, B, N_host, M_host, nodes_host ? nodes_host[0] : nullptr, q, eps, prec,
                               opt, stream);
    int64_t Mtot = 0;
    for (int i = 0; i < B; ++i) {
        if (M_host[i] < 0) return fail(FL_EINVAL, "fl_plan_batched_ptrs: need M_i >= 0");
        if (M_host[i] > 0 && (!nodes_host || !nodes_host[i]))
            return fail(FL_EINVAL, "fl_plan_batched_ptrs: nodes of a transform with M_i > 0 is NULL");
        Mtot += M_host[i];
    }
    if (Mtot > ((int64_t)1 << 31) - 1) return fail(FL_EUNSUPPORTED, "fl_plan_batched_ptrs: sum of M_i above 2^31 - 1");
    cudaStream_t st = (cudaStream_t)stream;
    double* cat = nullptr;   // the node sets concatenated, for planning only
    if (Mtot > 0) {
        FL_CUDA(cudaMalloc(&cat, Mtot * 2 * sizeof(double)), "cudaMalloc nodes");
        int64_t off = 0;
        for (int i = 0; i < B; ++i) {
            if (M_host[i] > 0) {
                const cudaError_t e = cudaMemcpyAsync(cat + 2 * off, nodes_host[i], M_host[i] * 2 * sizeof(double),
                                                      cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) {
                    cudaFree(cat);
                    return cuda_fail(e, "fl_plan_batched_ptrs: copy nodes");
                }
            }
            off += M_host[i];
        }
    }
    fl_status s = fl_plan_batched(out, B, N_host, M_host, cat, q, eps, prec, opt, stream);
    if (cat) {
        const cudaError_t e = cudaStreamSynchronize(st);
        cudaFree(cat);
        if (e != cudaSuccess && s == FL_OK) {
            fl_destroy(*out);
            *out = nullptr;
            return cuda_fail(e, "fl_plan_batched_ptrs: synchronise");
        }
    }
    return s;
}

fl_status fl_execute_batched_ptrs(fl_plan_t h, const void* const* c_host, void* const* f_host, void* stream) {
    if (!h || h->p.kind != 0 || !h->p.batched)
        return fail(FL_EINVAL, "fl_execute_batched_ptrs: not a batched Fourier-Laplace plan");
    Plan& p = h->p;
    const int B = (int)p.inst.size();
    if (!c_host || (p.M > 0 && !f_host)) return fail(FL_EINVAL, "fl_execute_batched_ptrs: NULL pointer array");
    for (int i = 0; i < B; ++i) {
        if (!c_host[i]) return fail(FL_EINVAL, "fl_execute_batched_ptrs: NULL coefficients");
        if (p.inst[i].M > 0 && !f_host[i]) return fail(FL_EINVAL, "fl_execute_batched_ptrs: NULL result");
    }
    const size_t cs = p.prec != FL_FP32 ? 16 : 8;
    cudaStream_t st = (cudaStream_t)stream;
    if (!p.d_stage_c) FL_CUDA(cudaMalloc(&p.d_stage_c, p.N * cs), "cudaMalloc staging");
    if (!p.d_stage_f && p.M > 0) FL_CUDA(cudaMalloc(&p.d_stage_f, p.M * cs), "cudaMalloc staging");
    if (!p.d_boff) {   // instance offsets, fixed for the plan
        std::vector<int64_t> off(2 * (B + 1));
        for (int i = 0; i < B; ++i) {
            off[i] = p.inst[i].noff;
            off[B + 1 + i] = p.inst[i].moff;
        }
        off[B] = p.N;
        off[2 * B + 1] = p.M;
        FL_CUDA(cudaMalloc((void**)&p.d_boff, off.size() * sizeof(int64_t)), "cudaMalloc offsets");
        FL_CUDA(cudaMemcpy(p.d_boff, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice),
                "copy offsets");
        FL_CUDA(cudaMalloc((void**)&p.d_bptr, 2 * (size_t)B * sizeof(void*)), "cudaMalloc pointer table");
    }
    // the caller's pointers (pageable host memory: the copy is staged before
    // the call returns, so the arrays may be reused at once)
    std::vector<const void*> ptrs(2 * (size_t)B, nullptr);
    for (int i = 0; i < B; ++i) {
        ptrs[i] = c_host[i];
        ptrs[B + i] = p.M > 0 ? f_host[i] : nullptr;
    }
    FL_CUDA(cudaMemcpyAsync(p.d_bptr, ptrs.data(), ptrs.size() * sizeof(void*), cudaMemcpyHostToDevice, st),
            "copy pointer table");
    FL_CUDA(launch_batch_pack(p, cs, true, st), "fl_execute_batched_ptrs: gather coefficients");
    FL_CUDA(forward_graphed(p, p.d_stage_c, p.d_stage_f, st), "fl_execute_batched_ptrs");
    if (p.M > 0) FL_CUDA(launch_batch_pack(p, cs, false, st), "fl_execute_batched_ptrs: scatter results");
    return FL_OK;
}

fl_status fl_get_info(fl_plan_t h, fl_info* info) {
    if (!h || !info) return fail(FL_EINVAL, "fl_get_info: NULL argument");
    const Plan& p = h->p;
    memset(info, 0, sizeof(*info));
    info->kind = p.kind;
    info->precision = p.prec;
    info->N = p.N;
    info->M = p.M;
    info->eps = p.eps;
    info->eps_laplace = p.eps_K;
    info->eps_fourier = p.eps_A;
    info->q = p.q;
    info->levels = p.levels;
    info->m_w = p.mw;
    info->sigma = 2;
    info->y1 = p.y1;
    info->xi1 = p.xi1;
    info->z0_nodes = p.z0_nodes;
    info->batch = p.batched ? (int)p.inst.size() : 1;
    if (p.kind == 0) {   // bands of all transforms: routes counted over the batch
        for (const BandHost& bh : p.bands) {
            if (bh.local == 0 || bh.dev.parent >= 0) continue;   // sub-bands count with their band
            if (bh.dev.route == 1) ++info->n_bands_fft;
            if (bh.dev.route == 2) ++info->n_bands_direct;
        }
    }
    const int nb_first = p.kind == 0 && !p.inst.empty() ? p.inst[0].levels + 1 : (int)p.bands.size();
    for (int b = 1; b < nb_first && b < (int)p.bands.size() && b < FL_MAX_LEVELS; ++b) {
        const BandHost& bh = p.bands[b];
        info->band_ell[b] = bh.ell;
        info->band_route[b] = bh.dev.route;
        info->band_nodes[b] = bh.nodes;
        info->band_K[b] = bh.dev.K;
        info->band_n[b] = bh.dev.n;
        info->band_parts[b] = bh.dev.nsub > 0 ? bh.dev.nsub : 1;
    }
    info->model_bytes = p.model_bytes;
    info->direct_bias = p.tuned_bias > 0 ? p.tuned_bias : p.direct_bias;
    info->scratch_bytes = p.scratch_bytes;
    info->variant = p.variant;
    info->kernel = p.kind == 1 ? p.lap_kernel : 0;
    info->n_bands_fused = (int)p.fused_bands;
    info->fused_entries = p.fused_entries;
    info->sigma_min = p.sigma_min;
    info->rhs_per_launch = p.rhs_per_launch;
    info->oversampling = p.sigma_mode;
    info->fuse_gather = p.fuse_mode;
    info->autotuned = p.tuned_rhs >= 0 ? 1 : 0;
    return FL_OK;
}

fl_status fl_set_timing(fl_plan_t h, int enable) {
    if (!h) return fail(FL_EINVAL, "fl_set_timing: NULL plan");
    Plan& p = h->p;
    for (Timer& t : p.timers) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    p.timers.clear();
    p.timing = enable != 0;
    p.launches = 0;
    return FL_OK;
}

fl_status fl_get_timing(fl_plan_t h, fl_timing* out) {
    if (!h || !out) return fail(FL_EINVAL, "fl_get_timing: NULL argument");
    Plan& p = h->p;
    memset(out, 0, sizeof(*out));
    for (Timer& t : p.timers) {
        cudaError_t e = cudaEventSynchronize(t.stop);
        if (e != cudaSuccess) return cuda_fail(e, "fl_get_timing");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, t.start, t.stop);
        if (e != cudaSuccess) return cuda_fail(e, "fl_get_timing");
        int slot = -1;
        for (int i = 0; i < out->n_kernels; ++i)
            if (t.name == out->name[i]) slot = i;
        if (slot < 0) {
            if (out->n_kernels >= FL_MAX_TIMED_KERNELS) continue;
            slot = out->n_kernels++;
            snprintf(out->name[slot], sizeof(out->name[slot]), "%s", t.name.c_str());
        }
        out->launches[slot] += 1;
        out->total_ms[slot] += ms;
        out->bytes[slot] += t.bytes;
    }
    out->total_launches = p.launches;
    return FL_OK;
}

void fl_destroy(fl_plan_t h) {
    if (!h) return;
    cudaDeviceSynchronize();
    delete h;
}

}  // extern "C"
