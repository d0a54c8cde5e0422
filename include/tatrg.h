/*
 * tatrg.h -- C ABI of the GB300 (sm_103a) Triad-ATRG library.
 *
 * The library coarse-grains the d-dimensional Ising partition function
 * Z = tTr prod_n T(n) (Sugimoto & Sasaki, arXiv:2412.14104, Sec. 3) with the Triad-ATRG
 * step of Sec. 2: the bond swap of Eq. 1 truncated by a randomized SVD, the oversampled
 * triad isometries and tensors of Eqs. 2-4, the squeezers of Eq. 5 and the O(r^2 chi^7)
 * contraction of Eqs. 6-7, followed by a re-split and normalisation.  Every stage runs in
 * the library's own CUDA kernels on one GPU.
 *
 * Conventions shared by all entry points
 *  - Status codes only; nothing throws across this boundary.  On an error the context
 *    keeps the message returned by tatrg_last_error().
 *  - "host" pointers are caller-owned CPU memory, read or written before the call returns.
 *    "device" pointers are caller-owned GPU memory on the current device; the call only
 *    enqueues work on the given stream unless it says it synchronises.
 *  - Tensors are dense row-major float64.  A site tensor is stored split as
 *    T[f; b] = sum_a A[f, a] s[a] B[a, b]: A has shape (D_0, ..., D_{d-1}, Da), s has Da
 *    entries, B has shape (Da, D_0, ..., D_{d-1}).  Leg position 0 is the direction the
 *    next step coarse-grains; after a step the leg order rotates left by one.
 *  - One context per host thread; a context is bound to the device current at creation.
 */
#ifndef TATRG_H
#define TATRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tatrg_ctx tatrg_ctx; /* opaque, library-owned */

typedef enum {
  TATRG_OK = 0,
  TATRG_EINVAL = 1,   /* bad argument (sizes, null pointer, unsupported d or precision) */
  TATRG_ENOMEM = 2,   /* device allocation failed */
  TATRG_ECUDA = 3,    /* a CUDA runtime or driver call failed */
  TATRG_ENUMERIC = 4, /* non-finite value, zero norm or non-convergent small solver */
  TATRG_ETIMEOUT = 5, /* a bounded device-side wait ran out */
  TATRG_ESTATE = 6,   /* calls in the wrong order (e.g. a step before init) */
  TATRG_ENOTIMPL = 7  /* the requested feature is not built */
} tatrg_status;

typedef enum { TATRG_ATRG = 0, TATRG_TRIAD = 1 } tatrg_method;

/* Arithmetic of the large contractions.  QR / SVD / eigen cores and ln Z stay float64. */
typedef enum {
  TATRG_FP64 = 0,   /* float64 CUDA-core GEMMs */
  TATRG_TF32X3 = 1, /* tcgen05 kind::tf32, operands split hi+lo, 3 products, FP32 accumulate */
  TATRG_BF16X3 = 2, /* tcgen05 kind::f16 with bf16 hi+lo split, 3 products, FP32 accumulate */
  TATRG_BF16X6 = 3, /* tcgen05 kind::f16 with bf16 hi+mid+lo split (the 24 bits of the float
                       nearest to each operand), the 6 products down to 2^-16 of hi*hi,
                       FP32 accumulate: the tensor time of TATRG_TF32X3 at float accuracy */
  TATRG_OZAKI = 4   /* float64-grade: each operand row (column) scaled by a power of two and
                       cut into five 7-bit integer slices (Ozaki et al. 2012), the 15 slice
                       products of weight >= 2^-28 on tcgen05 kind::f16 with exact FP32
                       sums over chunks of 512, combined in double-float: ~2^-36 relative
                       to the largest entries of the rows and columns involved */
} tatrg_precision;

typedef struct {
  int chi;        /* bond dimension (Sec. 2; Table 2 uses 38..54) */
  int r;          /* internal-line oversampling: triad lines carry r*chi (Fig. 1) */
  int q;          /* power iterations of every randomized SVD (Table 1) */
  int method;     /* tatrg_method */
  int precision;  /* tatrg_precision */
  unsigned long long seed; /* Philox key of all Gaussian sketches */
  int checkpoint_every;    /* unused (keep 0 or any value): the derivatives of tatrg_grad
                              are forward-mode tangents, which store nothing across steps,
                              so there is no reverse sweep to checkpoint */
  int split_from_step;     /* steps before this one run in FP64 whatever the precision */
  int split_stages;        /* bit mask of the stages whose large contractions use the split
                              precision: 1 swap, 2 triad, 4 squeezers, 8 contraction,
                              16 re-split; 0 means all */
  int profile;             /* 1: bracket every tensor-core GEMM with CUDA events and report
                              their device time in tatrg_step_info (tc_ms, tc_flops) */
  int sweep_workers;       /* temperatures tatrg_sweep runs concurrently (0: 8) */
  int early_precision;     /* split precision of the steps split_from_step .. late_from_step-1
                              (0: `precision`); e.g. TATRG_BF16X6 before TATRG_TF32X3 */
  int late_from_step;      /* first step that uses `precision` (0: split_from_step) */
} tatrg_params;

/* Create a context on `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * The context owns every device buffer it uses (stream-ordered allocations on that
 * stream).  Fails with EINVAL when chi < 1, r < 1, q < 0, or an enum is out of range. */
tatrg_status tatrg_create(const tatrg_params* params, void* cuda_stream, tatrg_ctx** out);

/* Build the Ising initial tensor of Sec. 3, T = sum_s e^{hs} prod_mu W[s,x_mu] W[s,x'_mu]
 * with W the symmetric square root of [[e^b, e^-b], [e^-b, e^b]] (the printed W without
 * its square roots is read as this), normalise it by its Frobenius norm c_0 and split it
 * exactly into A s B on the device.  d in {2, 3, 4}; beta > 0.  Resets the step count and
 * the ln Z accumulator to ln c_0.  Synchronises the context stream. */
tatrg_status tatrg_init_ising(tatrg_ctx* ctx, double beta, double h, int d);

/* Run `nsteps` coarse-graining steps (Sec. 2, Eqs. 1-7).  Each step halves the lattice
 * along the leg at position 0, normalises the new tensor by c_k = ||s'||_2 and adds
 * 2^-k ln c_k to the accumulator.  Returns after the last step's small host reads
 * (spectra needed for the rank cuts), so the call synchronises the stream.  Inside a
 * step the independent factorisations of the triad isometries (Eqs. 2-3) and of the
 * squeezer Grams (Eq. 5) run on short-lived host threads, each on a worker stream the
 * context owns; they start after the work already queued on the context's stream and the
 * context's stream waits for them, so the call keeps the stream semantics above. */
tatrg_status tatrg_rg_step(tatrg_ctx* ctx, int nsteps);

/* ln Z / V after the steps run so far: sum_k 2^-k ln c_k + 2^-N ln tTr T_N, where tTr
 * traces every forward leg with its own backward leg (a periodic lattice of 2^N sites).
 * Writes one double to a host pointer.  Synchronises. */
tatrg_status tatrg_lnZ(tatrg_ctx* ctx, double* lnZ_per_site);

/* Derivatives of the computed ln Z / V (tatrg_lnZ after the same steps) with respect to
 * beta and h: -dlnZ_dbeta is the internal energy per site (the beta derivative of beta f,
 * with the free energy f = -ln Z / (beta V) of Sec. 3), dlnZ_dh the magnetisation per site,
 * d2lnZ_dbeta2 the specific heat over beta^2.  The paper computes ln Z only; these are the
 * exact derivatives of the algorithm's output as a function of (beta, h), with every
 * sketch held fixed, obtained by forward-mode (tangent) propagation through all steps of
 * the run: one FP64 pass per first derivative (whatever the context's precision), and
 * the second derivative as the central difference (step 1e-6 max(1, beta)) of the exact
 * first derivative (two more passes).  The computed ln Z / V is piecewise smooth: where
 * kept singular values of different symmetry sectors cross, the ordered basis that later
 * sketches act on changes and ln Z / V jumps at the level of the truncation error; the
 * derivatives are those of the piece that contains (beta, h).  Needs a state made by
 * tatrg_init_ising; any of the three host pointers may be null (not all).  The passes are
 * independent and run concurrently, each on its own host thread and non-blocking stream,
 * after the work already queued on the context's stream; the call synchronises and leaves
 * the context's state untouched.  At h = 0 the h-derivative of the algorithm
 * is not smooth where symmetry-degenerate values split; use it at h != 0. */
tatrg_status tatrg_grad(tatrg_ctx* ctx, double* dlnZ_dbeta, double* dlnZ_dh,
                        double* d2lnZ_dbeta2 /* nullable */);

/* Independent runs over `nbeta` temperatures (host array `betas`), each `nsteps` steps
 * with the sketch replica index equal to its position in the array (so each result
 * equals a single run with that replica); writes ln Z / V for each to the host array
 * `lnZ_out`.  params.sweep_workers host threads run temperatures concurrently, each on
 * its own stream and device buffers.  The context's own state is left untouched.
 * Synchronises.  The first error of any run is returned. */
tatrg_status tatrg_sweep(tatrg_ctx* ctx, const double* betas, int nbeta, double h, int d,
                         int nsteps, double* lnZ_out);

/* The same temperature runs, also writing to the host array X_out (nullable, nbeta * nsteps
 * doubles) the order parameter X^(m) of tatrg_order_parameter at leg position d - 1 after
 * every step: X_out[i * nsteps + m - 1] is X^(m) of temperature i.  This is the temperature
 * scan of Sec. 3 that locates the transition point; the whole history is returned because
 * at h = 0 the two-fold degeneracy of the ordered phase is itself lost after enough steps
 * (rounding breaks the Z2 symmetry and the flow amplifies it), so X^(m) of the ordered
 * phase rises to 2 and later decays toward 1. */
tatrg_status tatrg_sweep_observables(tatrg_ctx* ctx, const double* betas, int nbeta, double h,
                                     int d, int nsteps, double* lnZ_out, double* X_out);

/* Order parameter of the transition point (Sec. 3, the definition of X^(m) after Gu & Wen):
 * A^(m)[k, l] = sum over every other leg x of T[.., x, k, ..; .., x, l, ..] with the forward
 * leg at position `leg` open as k and its backward leg as l, and
 * X = (Tr A^(m))^2 / Tr (A^(m))^2, written to a host double.  It counts the degeneracy of the
 * dominant sector: X -> 2 in the ordered phase of the Ising model at h = 0, X -> 1 in the
 * disordered phase.  After k steps leg position p is lattice direction (p + k) mod d.  One
 * FP64 contraction of the current state; synchronises.  EINVAL for a leg outside 0..d-1,
 * ESTATE before init, ENUMERIC when Tr (A^(m))^2 is zero or not finite. */
tatrg_status tatrg_order_parameter(tatrg_ctx* ctx, int leg, double* X);

/* Spectra of the last step, copied to a host array of capacity *n (on return *n holds
 * the count).  kind: 0 = s' (normalised, re-split), 1 = sigma of the bond swap,
 * 2 + (nu-1) = squeezer singular values of transverse leg position nu (1..d-1). */
tatrg_status tatrg_spectrum(const tatrg_ctx* ctx, int kind, double* out, int* n);

/* Copy the current state to host memory.  dims receives d+1 ints (D_0..D_{d-1}, Da);
 * *d receives d; A, s, B may be NULL to query the sizes only. */
tatrg_status tatrg_get_state(const tatrg_ctx* ctx, int* d, int* dims, double* A, double* s,
                             double* B);

/* Replace the state by host tensors (same layout as tatrg_get_state), with `step` steps
 * already taken and `partial_lnz` = sum_k 2^-k ln c_k so far.  Synchronises.  ENOMEM when
 * the device buffers cannot be allocated; ENUMERIC when A, s or B holds a non-finite
 * value.  On an error the previous state is kept. */
tatrg_status tatrg_set_state(tatrg_ctx* ctx, int d, const int* dims, const double* A,
                             const double* s, const double* B, int step, double partial_lnz);

/* Per-stage record of the last step (host struct). */
typedef struct {
  int step;            /* 1-based index of the step */
  int dims[5];         /* leg dims D_0..D_3 and Da after the step (unused legs = 0) */
  int swap_exact;      /* 1 when the swap used the exact SVD */
  double lnc;          /* ln c_k */
  double flops[5];     /* algorithmic flops: swap, triad, squeeze, contract, resplit */
  double ms[5];        /* device time of each stage (CUDA events) */
  double swap_gap;     /* (sigma_{Dg-1} - sigma_Dg) / sigma_0 at the swap cut (inf if none) */
  int tc_launches;     /* tcgen05 GEMM launches of the step on the context's stream; the
                          factorisations that run concurrently on worker streams (triad
                          isometries, squeezer factors) are counted in kernel_launches only,
                          since their event times include the GPU they share */
  int kernel_launches; /* all library kernel launches in the step */
  double tc_ms;        /* device time of the tc_launches (needs params.profile = 1) */
  double tc_flops;     /* their algorithmic flops, 2 M N K per contraction */
  double partial_lnz;  /* sum_k 2^-k ln c_k over k = 0 .. step (the input of tatrg_set_state) */
} tatrg_step_info;

tatrg_status tatrg_last_step_info(const tatrg_ctx* ctx, tatrg_step_info* out);

const char* tatrg_last_error(const tatrg_ctx* ctx);
void tatrg_destroy(tatrg_ctx* ctx);

/* ---------------------------------------------------------------------------------
 * Building blocks, exposed for parity tests and for callers that compose their own
 * networks.  All pointers are device pointers; work is enqueued on `cuda_stream`.
 * Errors of these calls are reported through tatrg_last_error(NULL).
 * --------------------------------------------------------------------------------- */

/* Gaussian sketch used by every randomized SVD (Table 1: RSVD with q iterations): element
 * e of the row-major rows x cols output is z_{e mod 2} of the Box-Muller pair made from
 * Philox4x32-10 with counter (lo32(e/2), hi32(e/2), replica, hi32(seed)) and key
 * (lo32(seed), stream_id).  Writes rows*cols doubles to `out`. */
tatrg_status tatrg_gaussian(unsigned long long seed, uint32_t stream_id, uint32_t replica,
                            int64_t rows, int64_t cols, double* out, void* cuda_stream);

/* A tensor contraction C[m, n] = alpha sum_k A[m, k] B[k, n] + beta C[m, n] whose m, n
 * and k are each up to 4 modes with their own element strides (this is how the
 * contractions of Eqs. 1-7 are expressed without transposes).  Mode i of m has extent
 * m_ext[i], stride m_sA[i] in A and m_sC[i] in C; modes are listed outermost first and
 * unused ones have extent 1.  precision selects the FP64 or a split tensor-core path. */
typedef struct {
  int64_t m_ext[4], m_sA[4], m_sC[4];
  int64_t n_ext[4], n_sB[4], n_sC[4];
  int64_t k_ext[4], k_sA[4], k_sB[4];
  double alpha, beta;
} tatrg_contraction;

tatrg_status tatrg_contract(const tatrg_contraction* c, int precision, const double* A,
                            const double* B, double* C, void* cuda_stream);

/* tatrg_contract with B the Gaussian sketch of tatrg_gaussian (seed, stream_id, replica;
 * element B[k, n] is sketch element number sum_i k_i k_sB[i] + sum_i n_i n_sB[i]), generated
 * while the tensor-core operand is packed and never stored: the random test matrix of the
 * randomized SVD (Halko et al. Alg. 4.4, used for the bond swap of Eq. 1, Table 1) drawn in
 * the contraction's operand producer.  Only for the split precisions (precision 1, 2 or 3,
 * where Box-Muller runs in float arithmetic: the values equal tatrg_gaussian's rounded to
 * float) and contractions large enough for the tensor cores (EINVAL otherwise).  The
 * result equals tatrg_contract on that sketch rounded to float, stored.  Synchronises. */
tatrg_status tatrg_contract_sketch(const tatrg_contraction* c, int precision, const double* A,
                                   unsigned long long seed, uint32_t stream_id, uint32_t replica,
                                   double* C, void* cuda_stream);

/* Orthonormal basis of the columns of the row-major m x n matrix Y (m >= n): Y = Q R with
 * Q^T Q = 1 and R upper triangular with a non-negative diagonal when Y has full column
 * rank (CholeskyQR2 with shift); a rank-deficient Y returns k < n columns spanning its
 * range and R of shape k x n.  Q must hold m*n doubles, R n*n.  *k (host) receives the
 * column count.  Synchronises the stream. */
tatrg_status tatrg_orth(int precision, int64_t m, int64_t n, const double* Y, double* Q,
                        double* R, int* k, void* cuda_stream);

/* Thin SVD of a row-major m x n matrix (m >= n, n <= 1024) by one-sided Jacobi:
 * A = U diag(S) V^T with S descending.  U: m x n, S: n, V: n x n (row-major, columns are
 * the right singular vectors).  Synchronises the stream. */
tatrg_status tatrg_svd(int64_t m, int64_t n, const double* A, double* U, double* S, double* V,
                       void* cuda_stream);

/* The same thin SVD as tatrg_svd, for callers that cannot allocate device memory: code
 * that runs while another allocator owns the whole device budget (a framework's caching
 * pool, a fixed reservation), or code where the implicit synchronisation of cudaMalloc /
 * cudaFree is not allowed.  The paper has no counterpart; this is a property of the
 * library.  No memory is allocated: the workspace is one fixed device array of 2 MiB
 * (262144 doubles) that every GPU loading the library keeps until the process exits, so
 * the size limit is (m + N + 2) * N + 3 <= 262144 with N = n rounded up to even: for
 * example n = 144 allows m <= 1674, n = 256 allows m <= 765, n = 2 allows m <= 131066.
 * Larger inputs return TATRG_EINVAL.  The first call on a device looks up that array's
 * device address; make that first call before any stream capture on the device.  All
 * calls share the array: calls whose work overlaps on the GPU race; each call rewrites
 * every part of the workspace it reads.  Pointers are device pointers with the layout of
 * tatrg_svd; the call synchronises the stream.  Errors go to tatrg_last_error(NULL). */
tatrg_status tatrg_svd_noalloc(int64_t m, int64_t n, const double* A, double* U, double* S,
                               double* V, void* cuda_stream);

/* Raw words of the sketch generator (A10; the RSVD test matrices of Table 1): for counter
 * blocks p = first .. first + npairs - 1, the four 32-bit outputs of Philox4x32-10 with
 * counter (lo32(p), hi32(p), replica, hi32(seed)) and key (lo32(seed), stream_id), written
 * to the device array `out` (4 * npairs words, word j of block p at 4 (p - first) + j;
 * 16-byte aligned); p wraps modulo 2^64.  These are the integers every Gaussian sketch of
 * tatrg_gaussian and of the operand packer is made from; they are exposed so the stream
 * can be compared bit for bit.  EINVAL when npairs < 0 or out is null or unaligned. */
tatrg_status tatrg_philox_words(unsigned long long seed, uint32_t stream_id, uint32_t replica,
                                uint64_t first, int64_t npairs, uint32_t* out, void* cuda_stream);

/* Time limit of the grid-wide barrier between the rounds of the cooperative Jacobi SVD
 * (every core SVD of the step with n >= 32), in nanoseconds, for the current device; the
 * default is 2e9 (2 s).  When a block waits longer, every block of that launch returns
 * and the SVD reports TATRG_ETIMEOUT; the context stays usable.  The paper has no
 * counterpart: this is the library's failure detection, and the setter exists so that
 * a test can make the wait run out (a limit of 0 expires at the first wait).  It does not
 * change the bounded waits of the tensor-core pipeline.  EINVAL for a negative limit. */
tatrg_status tatrg_set_barrier_limit_ns(long long limit_ns);

/* Launch policy of the split-precision tensor-core contractions (3xTF32, BF16x3, BF16x6;
 * the contractions of Eqs. 1-7) for the whole process.  Tile forms: single CTAs (one
 * 128 x 128 output tile per CTA); CTA pairs (cta_group::2: one tensor-core MMA of
 * 256 x 128 on two SMs, each holding half of the B tile); multicast clusters (two CTAs
 * with a 128 x 128 tile each, stacked in M, each loading half of the shared B tile and
 * multicasting it to both).  mode 0 (the default) lets the autotuner pick the form and the
 * split of K per contraction shape, with single CTAs for untuned shapes; 1 takes CTA pairs
 * and 2 multicast clusters wherever they apply (M >= 1024 output rows); -1 never takes the
 * two-CTA forms.  Results agree to the split form's rounding whatever the form.  The paper
 * has no counterpart: the setter exists so that tests and measurements can choose the
 * form.  EINVAL for any other value. */
tatrg_status tatrg_set_cta_pairs(int mode);

#ifdef __cplusplus
}
#endif
#endif /* TATRG_H */
