/*
 * fl.h -- C ABI of the GB300 fast Fourier-Laplace transform library (libfl.so).
 *
 * Kunis & Melzer, "Fast evaluation of real and complex exponential sums"
 * (arXiv 1606.03255).  The library evaluates
 *
 *   f_j = sum_{k=0}^{N-1} c_k exp(2 pi i k w_j),   Im w_j >= 0,   j < M,
 *
 * i.e. the polynomial sum_k c_k z^k at the nodes z_j = exp(2 pi i w_j) of the
 * closed unit disk (Section 4, eq. (4.1) with exponents xi_k = k and the polar
 * split (4.2); this ABI numbers coefficients from 0 where the paper numbers
 * them from 1), by Algorithm 2 of the paper, and the real discrete Laplace
 * transform f_j = sum_k c_k exp(-s_j t_k) (Section 3, eq. (3.2)) by
 * Algorithm 1.  Every step runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions shared by every call:
 *   - All pointers named *_dev are device pointers (e.g. from torch tensors);
 *     *_host pointers are host memory (pinned memory gives overlapped copies).
 *     The caller owns every buffer it passes; the plan owns its own scratch.
 *   - Complex arrays are interleaved (re, im).  The element type follows the
 *     plan's precision: FL_FP32 -> (float, float) (complex64),
 *     FL_FP64 and FL_FP64_FF -> (double, double) (complex128).  Nodes are
 *     always float64.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  fl_execute / fl_adjoint / fl_laplace_real are asynchronous on
 *     it; planning synchronises it.
 *   - Errors are returned as fl_status, never raised or aborted on; a message
 *     is kept per thread and read with fl_last_error().
 *   - A plan may be executed any number of times; one plan must not be used by
 *     two host threads at the same time.
 */
#ifndef FL_H
#define FL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fl_plan_s *fl_plan_t;

typedef enum {
    FL_OK = 0,
    FL_EINVAL = 1,        /* invalid argument (sizes, eps, Im w < 0, NaN ...) */
    FL_ENOMEM = 2,        /* device or host allocation failed                 */
    FL_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed      */
    FL_ETIMEOUT = 4,      /* reserved: no kernel of this library waits on
                             another (every launch's work is independent of
                             the others in flight), so no call returns it    */
    FL_EUNSUPPORTED = 5   /* size or parameter outside what is implemented    */
} fl_status;

/* FL_FP64_FF: the FP64-accuracy form with complex128 c and f whose band-grid
 * FFTs run in float pairs (hi + lo, about 48 significant bits from FP32
 * arithmetic, which this part issues at 64 times its FP64 rate); the
 * coefficient weights and twiddles are rounded once from FP64 to pairs, and
 * the window gather, barycentric recombination and direct bands also run in
 * pairs (exponential, sincospi, square root and division written for pairs),
 * with the phases n x mod 1 reduced exactly in double.  fl_plan, fl_plan_ex
 * and fl_plan_batched accept it, with fl_execute, fl_execute_host and
 * fl_execute_batched, and on single plans fl_execute_deriv and fl_grad_w
 * (Algorithm 2 on the k-weighted coefficients 2 pi i k c_k, formed in double
 * and rounded to pairs) and fl_adjoint and fl_transposed (the spreading,
 * direct bands and the final weighting sum_s D[s][k] b_s in double, the
 * spread grids rounded to pairs for the sign -1 FFTs in pairs).  The other
 * plan calls reject it with FL_EINVAL. */
typedef enum { FL_FP32 = 0, FL_FP64 = 1, FL_FP64_FF = 2 } fl_precision;

#define FL_MAX_LEVELS 128

/* Plan parameters and per-band sizes, filled by fl_get_info. */
typedef struct {
    int kind;                 /* 0 = Fourier-Laplace (Alg. 2), 1 = Laplace (Alg. 1) */
    int precision;            /* fl_precision */
    int64_t N, M;
    double eps;               /* target accuracy: ||f - f~||_inf <= eps ||c||_1 */
    double eps_laplace;       /* accuracy given to the Laplace factor (eps/3 for Alg. 2) */
    double eps_fourier;       /* accuracy given to each NFFT (eps/3) */
    int q;                    /* interpolation rank (Definition 3.2) */
    int levels;               /* number of dyadic levels, the paper's M (Definition 3.2) */
    int m_w;                  /* Kaiser-Bessel window half-width (taps = 2 m_w) */
    int sigma;                /* oversampling of unsplit band grids (2; see sigma_min) */
    double y1, xi1;           /* interval ends of Definition 3.2 */
    int64_t z0_nodes;         /* nodes with |z| < eps (returned as c_0) */
    int batch;                /* transforms in the plan (fl_plan_batched), else 1 */
    int n_bands_fft;          /* bands evaluated with an NFFT (all transforms) */
    int n_bands_direct;       /* bands evaluated by the direct-sum kernel (all transforms) */
    /* per band b = 1..levels of the (first) transform (index 0 unused): */
    int band_ell[FL_MAX_LEVELS];      /* l_m (first interpolated frequency band) */
    int band_route[FL_MAX_LEVELS];    /* 0 empty, 1 NFFT, 2 direct */
    int64_t band_nodes[FL_MAX_LEVELS];
    int64_t band_K[FL_MAX_LEVELS];    /* frequencies with nonzero weight */
    int64_t band_n[FL_MAX_LEVELS];    /* FFT length (oversampled grid) */
    double model_bytes;       /* algorithmic HBM bytes of one fl_execute */
    double direct_bias;       /* route bias in use (the autotuner's choice if tuned) */
    double scratch_bytes;     /* device memory owned by the plan */
    int variant;              /* fl_options.variant in use */
    int kernel;               /* Laplace plans: the fl_kernel */
    int n_bands_fused;        /* bands whose window gather runs inside pass 2 (fuse_gather) */
    int64_t fused_entries;    /* their (node, pass-2 row block) entries */
    double sigma_min;         /* smallest oversampling n / K_p of the plan's grids (2 if none split) */
    int band_parts[FL_MAX_LEVELS];    /* NFFTs per band (1, or P sub-bands of band_n points each) */
    int rhs_per_launch;       /* grids per four-step launch pair (0 = all of a size) */
    int oversampling;         /* fl_options.oversampling the plan was built with */
    int fuse_gather;          /* fl_options.fuse_gather the plan was built with */
    int autotuned;            /* 1 if the settings above and direct_bias came from
                                 the autotuner (fl_options.autotune)            */
} fl_info;

/* Per-kernel timing gathered while timing is enabled (fl_set_timing). */
#define FL_MAX_TIMED_KERNELS 16
typedef struct {
    int n_kernels;
    char name[FL_MAX_TIMED_KERNELS][32];
    int64_t launches[FL_MAX_TIMED_KERNELS];
    double total_ms[FL_MAX_TIMED_KERNELS];
    double bytes[FL_MAX_TIMED_KERNELS];   /* algorithmic bytes summed over launches */
    int64_t total_launches;               /* every kernel launched by execute calls */
} fl_timing;

/*
 * fl_plan -- plan Algorithm 2 (Section 4) for N coefficients and M nodes.
 *   nodes_dev : device, M x {Re w_j, Im w_j} float64, Im w_j >= 0, finite.
 *               Read during planning only (the plan keeps a sorted copy).
 *   q         : interpolation rank; 0 = from eps by Definition 3.2,
 *               q = ceil(1/2 + log_4(3/eps)) (the Laplace factor gets eps/3,
 *               Lemma 4.1).
 *   eps       : target accuracy in (0, 1); the result satisfies
 *               max_j |f_j - f~_j| <= eps * sum_k |c_k| (Theorem 4.3) up to
 *               the rounding of the chosen precision.
 *   prec      : FL_FP32 (grids, FFT and recombination in float; phases and
 *               barycentric differences in double), FL_FP64, or FL_FP64_FF
 *               (FFTs in float pairs, the rest in double; see fl_precision).
 * Returns FL_EINVAL for N < 1, M < 0, eps outside (0, 1), q outside [0, 40] or
 * a node with Im w < 0 or a non-finite part; FL_EUNSUPPORTED for N > 2^23.
 * On failure *out is NULL.
 */
fl_status fl_plan(fl_plan_t *out, int64_t N, int64_t M, const double *nodes_dev,
                  int q, double eps, fl_precision prec, void *stream);

/* Planning options (fl_plan_ex). */
typedef struct {
    int route;            /* how each non-empty band is evaluated:
                             0 = by estimated cost (default): an NFFT with q
                                 right-hand sides, or the direct sum of eq. (4.1)
                                 over the band's frequencies when it has few nodes;
                             1 = every band by NFFT (Algorithm 2 as printed);
                             2 = every band by the direct sum                      */
    double direct_bias;   /* multiplies the direct-sum cost in route 0 (0 = 1.0)  */
    int rhs_per_launch;   /* grids of one size per four-step launch pair; small
                             values keep the intermediate in L2 (0 = all)         */
    int use_graph;        /* fl_execute: 1 = capture the launches in a CUDA graph
                             on the first call and replay it (re-captured when the
                             buffers or the stream change; not on the legacy
                             default stream).  fl_plan_batched: graphs are on
                             unless this is -1.  0 = plain launches.             */
    int autotune;         /* 1 = with route 0, plan the workload for several
                             values of direct_bias, time an execute of each on
                             `stream` and keep the fastest (cached per workload
                             signature for the process); 0 = off              */
    int variant;          /* weights of an interpolated band Y_m:
                             0 = Algorithm 2 (default): Chebyshev interpolation
                                 in y and in the frequency (Lemma 4.2, q from
                                 Definition 3.2);
                             1 = one-sided: interpolation in y only, each
                                 frequency k weighted by the exact
                                 exp(-y_s k) at the band's Chebyshev points y_s
                                 (the first term of the proof of Theorem 3.1);
                                 q = 0 then means the smallest q with
                                 2 q^q e^-q / (4^q q!) <= eps/3, the
                                 per-entry bound of that interpolation.       */
    int fuse_gather;      /* FL_FP32 forward transforms (fl_execute, the
                             derivative and gradient calls, batches): the
                             window gather of a band computed inside the second
                             pass of its grid's FFT, so that the grid is never
                             written to memory -- each node's taps are summed
                             per pass-2 tile into partial sums that the gather
                             recombines (the plan keeps the node/tile lists):
                             0 = for grids above 4096 points whose nodes are
                                 few for the grid (by estimated bytes; default);
                             1 = never; 2 = for every grid above 4096 points. */
    int oversampling;     /* FL_FP32 plans whose gather can be fused (above)
                             and FL_FP64 plans (whose sub-bands are gathered
                             from their grids): the oversampling sigma of a
                             band's NFFT.
                             0 = from the tolerance by estimated cost
                                 (default): a band with K frequencies may be
                                 evaluated as P NFFTs over contiguous ranges of
                                 about K/P frequencies on power-of-two grids of
                                 sigma K/P points, 1.25 <= sigma < 2, with the
                                 window half-width m_w that meets eps/3 at the
                                 smallest sigma used; a split is admitted only
                                 while the deconvolution's gain
                                 Phi(0)/Phi(1/(2 sigma)), which scales the
                                 grids' rounding, stays <= 32 in FP32 (so
                                 sigma >= ~1.5) and <= 2^47 eps/3 in FP64
                                 (sigma >= 1.75 at eps = 1e-12); float-pair
                                 plans keep sigma = 2;
                             1 = sigma = 2 for every band (one NFFT each);
                             2 = every eligible band split to its fewest grid
                                 points under the same limits, whatever the
                                 cost.                                        */
    int shared_nodes;     /* fl_plan_batched only: 1 = every transform takes
                             the same M_0 nodes (nodes_dev holds M_0 rows and
                             every M_i must equal M_0; N_i may differ).  The
                             nodes are classified and sorted once per distinct
                             N_i, and transforms of equal N_i share one weight
                             table D; 0 = one node set per transform.         */
} fl_options;

/*
 * fl_plan_ex -- fl_plan with options (NULL = defaults, i.e. fl_plan).
 * Returns FL_EINVAL for an invalid option value.
 */
fl_status fl_plan_ex(fl_plan_t *out, int64_t N, int64_t M, const double *nodes_dev,
                     int q, double eps, fl_precision prec, const fl_options *opt,
                     void *stream);

/*
 * fl_plan_batched -- one plan for B independent transforms of sizes
 * N_host[i] x M_host[i] (host arrays), i < B, with the same eps, q and
 * precision.  nodes_dev holds the nodes of transform 0, then 1, ... (sum M_i
 * rows of {Re w, Im w}, float64), or with fl_options.shared_nodes the M_0
 * rows that every transform shares.  Every kernel launch of fl_execute_batched
 * covers all B transforms (one global band table; the four-step FFTs of all
 * transforms of one grid size share a launch), and the launches are captured
 * in a CUDA graph and replayed (see fl_options.use_graph).  Forward only.
 */
fl_status fl_plan_batched(fl_plan_t *out, int B, const int64_t *N_host, const int64_t *M_host,
                          const double *nodes_dev, int q, double eps, fl_precision prec,
                          const fl_options *opt, void *stream);

/*
 * fl_execute_batched -- all transforms of a batched plan: c_dev holds the
 * coefficients of transform 0, 1, ... (sum N_i complex), f_dev receives the
 * results in the same order (sum M_i complex).
 */
fl_status fl_execute_batched(fl_plan_t p, const void *c_dev, void *f_dev, void *stream);

/*
 * fl_plan_batched_ptrs -- fl_plan_batched with one node array per transform:
 * nodes_host is a host array of B device pointers, entry i holding M_i rows
 * of {Re w, Im w} (NULL allowed where M_i = 0); with
 * fl_options.shared_nodes only entry 0 is read (the M_0 shared rows).  The
 * node sets are copied into one temporary device array for planning, which
 * is freed before the call returns (the call synchronises `stream`).
 */
fl_status fl_plan_batched_ptrs(fl_plan_t *out, int B, const int64_t *N_host, const int64_t *M_host,
                               const double *const *nodes_host, int q, double eps, fl_precision prec,
                               const fl_options *opt, void *stream);

/*
 * fl_execute_batched_ptrs -- fl_execute_batched on per-transform buffers:
 * c_host and f_host are host arrays of B device pointers (transform i: N_i
 * and M_i complex of the plan's precision; f entries may be NULL where
 * M_i = 0).  One kernel gathers the coefficients into the plan's staging
 * array, the batched transform runs on it, and one kernel scatters the
 * results; the pointer arrays are read before the call returns.
 * Asynchronous on `stream`.
 */
fl_status fl_execute_batched_ptrs(fl_plan_t p, const void *const *c_host, void *const *f_host,
                                  void *stream);

/*
 * fl_execute -- f~ ~= C c with C = (z_j^k), Algorithm 2.
 *   c_dev : device, N complex (plan precision).
 *   f_dev : device, M complex (plan precision), fully overwritten.
 * Asynchronous on `stream`.
 */
fl_status fl_execute(fl_plan_t p, const void *c_dev, void *f_dev, void *stream);

/*
 * fl_execute_deriv -- f'_j = sum_k (2 pi i k) c_k z_j^k = d f / d w at w_j, the
 * same Algorithm 2 applied to the k-weighted coefficients (the derivative of
 * eq. (4.1) in w).  Same arguments and accuracy scale as fl_execute, with
 * ||c||_1 replaced by sum_k 2 pi k |c_k|.
 */
fl_status fl_execute_deriv(fl_plan_t p, const void *c_dev, void *fprime_dev, void *stream);

/*
 * fl_grad_w -- gw_j = r_j * conj(f'_j), f'_j = sum_k (2 pi i k) c_k z_j^k: the
 * gradient of a real loss with respect to the nodes w_j, given the upstream
 * gradient r = dL/dRe f + i dL/dIm f (the chain rule for the holomorphic map
 * w -> f(w) of eq. (4.1)).  fl_execute_deriv with the product fused into its
 * last kernel.  c_dev: N complex; r_dev, gw_dev: M complex (plan precision).
 * Z^0 nodes get 0.
 */
fl_status fl_grad_w(fl_plan_t p, const void *c_dev, const void *r_dev, void *gw_dev,
                    void *stream);

/*
 * fl_execute_host -- fl_execute on host buffers: copies c_host (N complex) to
 * the device, executes, copies the result to f_host (M complex) and
 * synchronises `stream`.  Staging buffers are owned by the plan.
 */
fl_status fl_execute_host(fl_plan_t p, const void *c_host, void *f_host, void *stream);

/*
 * fl_adjoint -- c_out = C^* r, (C^* r)_k = sum_j conj(z_j)^k r_j, the adjoint
 * of Algorithm 2 (Section 4, the remark after Algorithm 2): every step of the
 * forward transform transposed and conjugated.
 *   r_dev     : device, M complex.   c_out_dev : device, N complex, overwritten.
 * Accuracy: |c_out - C^* r|_inf <= eps * sum_j |r_j| up to rounding.
 */
fl_status fl_adjoint(fl_plan_t p, const void *r_dev, void *c_out_dev, void *stream);

/*
 * fl_transposed -- g_k = sum_j ghat_j z_j^k for k = 0 .. N-1, i.e. C^T ghat:
 * the evaluation of g(xi) = sum_j ghat_j z_j^xi at the integer exponents
 * xi = k that the remark after Algorithm 2 (Section 4) obtains from the
 * adjoint algorithms; computed as conj(C^* conj(ghat)).  On a plan of
 * fl_plan_xi: g_k = sum_j ghat_j z_j^{xi_k} at the plan's real exponents, in
 * their original order (fl_adjoint likewise returns sum_j conj(z_j^{xi_k}) r_j).
 *   g_dev   : device, M complex (plan precision).
 *   out_dev : device, N complex, overwritten.
 * Accuracy as fl_adjoint.  The plan keeps an M-element staging buffer
 * (allocated on the first call).  Not for batched plans (FL_EUNSUPPORTED).
 */
fl_status fl_transposed(fl_plan_t p, const void *g_dev, void *out_dev, void *stream);

/*
 * fl_plan_xi -- plan the generalised polynomial of eq. (4.1) with real
 * exponents: f_j = sum_k c_k z_j^{xi_k} = sum_k c_k exp(2 pi i xi_k w_j),
 * xi_k >= 1 (the paper's xi_k in [1, N]).  Algorithm 2 with the bands and
 * weights evaluated at the exponent values (xi_1 = max xi_k) and every band's
 * Fourier factor computed by an NNFFT (nonequispaced in time and frequency,
 * as the proof of Theorem 4.3 notes): the exponents are spread onto a
 * frequency grid of spacing 1/2 with a Kaiser-Bessel window, followed by an
 * NFFT at x/2 and the division by the window's transform.  Each band is
 * centred on its exponent range; its NFFT keeps the half-size bandwidth when
 * only the window margin (at most m_w + 3 frequencies) overflows it and the
 * Kaiser-Bessel aliasing term grows by at most 1 %.
 *   xi_dev    : device, N float64 exponents >= 1 (any order; read at planning).
 *   nodes_dev : device, M x {Re w, Im w}; |Re w| <= 1/2 (principal branch of
 *               z^xi, the negative real axis Re w = +-1/2 as a one-sided
 *               limit), Im w >= 0.
 *   q, eps, prec : as fl_plan (each NNFFT gets eps/3).
 * Nodes with |z| < eps return 0 (every term is below eps |c_k| there).
 * Calls: fl_execute / fl_execute_host (forward), fl_adjoint and fl_transposed
 * (every step transposed: spreading at x/2 with the conjugate epilogue, FFTs
 * of sign -, the outer deconvolution and the frequency window gathered back to
 * each exponent); the derivative and gradient calls return FL_EUNSUPPORTED.
 * Returns FL_EINVAL for an exponent below 1 or not finite and for a node
 * outside the range above, FL_EUNSUPPORTED for N > 2^22.
 */
fl_status fl_plan_xi(fl_plan_t *out, int64_t N, const double *xi_dev, int64_t M,
                     const double *nodes_dev, int q, double eps, fl_precision prec, void *stream);

/*
 * fl_plan_laplace -- plan Algorithm 1 (Section 3) for the real discrete Laplace
 * transform f_j = sum_k c_k exp(-s_j t_k).
 *   t_dev : device, N float64 frequencies t_k >= 0.
 *   s_dev : device, M float64 nodes s_j >= 0.
 *   q, eps: as Definition 3.2 (the whole eps goes to the Laplace factor).
 *   prec  : FL_FP64, or FL_FP32 (float moments/evaluation, double weights).
 * Data is real: c and f are float64 for FL_FP64 and float32 for FL_FP32.
 */
fl_status fl_plan_laplace(fl_plan_t *out, int64_t N, int64_t M, const double *t_dev,
                          const double *s_dev, int q, double eps, fl_precision prec,
                          void *stream);

/* Kernels of fl_plan_kernel. */
typedef enum {
    FL_KERNEL_LAPLACE = 0,        /* exp(-s t) by Algorithm 1 (= fl_plan_laplace)     */
    FL_KERNEL_EXP_GENERAL = 1,    /* exp(-s t) by the generalised Algorithm 1         */
    FL_KERNEL_BESSEL_K_HALF = 2   /* K_{1/2}(s t) = sqrt(pi / (2 s t)) exp(-s t),
                                     s, t > 0 (the example after that theorem)       */
} fl_kernel;

/*
 * fl_plan_kernel -- plan f_j = sum_k c_k kappa(s_j, t_k) for an asymptotically
 * smooth kernel by the generalised Algorithm 1 (Section 3, the theorem after
 * Algorithm 1): every block Y_m x Omega_l, 1 <= m, l <= M - 1, interpolated
 * with q Chebyshev points per side, the near fields Y_M (all frequencies) and
 * Omega_M (all nodes) summed directly, M = ceil(log2(y_1 xi_1 N / eps)) + 1
 * (y_1 = max s_j, xi_1 = max t_k).
 *   kernel : fl_kernel; FL_KERNEL_LAPLACE forwards to fl_plan_laplace.
 *   q      : 0 = the smallest q whose block bound from the proof of Theorem 3.1,
 *            C mu^q q^nu 2^(1-2q) (2 + (2/pi) ln q) (y_1 xi_1 / 4^(M-1))^-s
 *            (exp: C = 1, s = 0; K_1/2: C = sqrt(pi/2), s = 1/2; mu = 1, nu = 0),
 *            is at most eps; else 1 .. 64.
 *   t_dev, s_dev, eps, prec : as fl_plan_laplace.
 * Execute with fl_laplace_real.  Cost: O(N q + M q + (M - 1)^2 q^2), plus the
 * direct near fields (|Y_M| N + M |Omega_M| kernel evaluations).
 * Returns FL_EINVAL for a negative, non-finite (or, for K_1/2, zero) node,
 * FL_EUNSUPPORTED for a rank above 64 or more than 127 levels.
 */
fl_status fl_plan_kernel(fl_plan_t *out, int kernel, int64_t N, int64_t M, const double *t_dev,
                         const double *s_dev, int q, double eps, fl_precision prec, void *stream);

/* fl_laplace_real -- f~ ~= K c (Algorithm 1, or the generalised Algorithm 1
 * of a fl_plan_kernel plan), c_dev N reals, f_dev M reals. */
fl_status fl_laplace_real(fl_plan_t p, const void *c_dev, void *f_dev, void *stream);

/*
 * fl_laplace_real_noalloc -- the real Laplace transform of fl_plan_laplace +
 * fl_laplace_real in one call that allocates no device memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate at
 * the point where they need the transform -- code running inside another
 * framework's memory pool that forbids outside allocations, real-time loops
 * where cudaMalloc (which can synchronise the whole device) is not allowed,
 * or a device that is already full.
 *   t_dev, s_dev, c_dev, f_dev, q, eps, prec : as fl_plan_laplace and
 *               fl_laplace_real (c and f real, float64 for FL_FP64, float32
 *               for FL_FP32); the result is theirs up to rounding (the
 *               planned call sums the moments in band order).
 * Scratch: a fixed static device array of 2 MiB, held by every GPU that loads
 * libfl.so until the process exits.  Its use depends on the number of levels
 * and on q only, not on N or M (the partial moment sums of the largest block
 * count are reserved whatever N is): about 1 KiB (FP64) or 0.5 KiB (FP32) per
 * entry of the (levels + 1) x (q + 1) moment table.  A problem that needs more
 * returns FL_EUNSUPPORTED with the bytes needed in fl_last_error().
 * The first call on each device does a one-time set-up (it looks up the
 * array's device address).  The call synchronises `stream` once (it reads max t and max s back to choose
 * the levels).  Every call on a device shares the one array, which keeps the
 * last call's contents: calls that overlap on the GPU (two streams, two host
 * threads) race and give wrong results, so serialise them.
 */
fl_status fl_laplace_real_noalloc(int64_t N, int64_t M, const double *t_dev,
                                  const double *s_dev, const void *c_dev, void *f_dev,
                                  int q, double eps, fl_precision prec, void *stream);

/* Plan parameters and sizes (host call, no device work). */
fl_status fl_get_info(fl_plan_t p, fl_info *info);

/* Enable (1) or disable (0) per-kernel CUDA-event timing; resets counters. */
fl_status fl_set_timing(fl_plan_t p, int enable);

/* Read the timing counters (synchronises the events recorded so far). */
fl_status fl_get_timing(fl_plan_t p, fl_timing *out);

/* Release the plan and its device memory (synchronises the device). */
void fl_destroy(fl_plan_t p);

/* Message of the last failing call on this host thread ("" if none). */
const char *fl_last_error(void);

/* Library version string. */
const char *fl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FL_H */
