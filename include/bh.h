/*
 * bh.h -- C ABI of libbh: ball-harmonic expansion and rotational matching on one GB300 GPU.
 *
 * The library computes the two data-parallel stages of "Beyond Exhaustive Sampling: Efficient
 * Rotational Matching via Ball Harmonics":
 *
 *   1. expansion of voxel volumes into ball-harmonic coefficients f_hat_klm on the basis
 *      psi_klm = c_lk j_l(lambda_lk r) Y_l^m(theta, phi) chi_[0,1)(r)   (Sec. II-A), and
 *   2. maximisation over rotations g of the rotational cross-correlation of Eq. 2 at shift s = 0,
 *      C(g) = sum_{l<=L} sum_{m,m'} xi_{l,m,m'} D^l_{m,m'}(g), with its closed-form gradient,
 *      multi-start gradient ascent and frequency marching (Sec. II-C); the closed-form Hessian and
 *      damped Newton steps, and candidate starts from the local maxima of the lowest band on a
 *      rotation grid (Sec. III); and the search over a grid of integer shifts (Eq. 1).
 *
 * Conventions (all calls):
 *   - Every call returns an int status: BH_OK (0), BH_PENDING (1, serving poll only) or a
 *     negative BH_ERR_* code.  bh_last_error() returns a thread-local description of the last
 *     failure on the calling thread.
 *   - Array arguments documented as "device" are device pointers owned by the caller (for
 *     example allocated by PyTorch); the library never frees them.  "host" arrays are ordinary
 *     host memory.  Handles (bh_plan, bh_grid, bh_server) are created and destroyed by the
 *     library.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Device work is
 *     enqueued asynchronously on it; the call returns once the work is queued.  Argument errors
 *     are reported before anything is enqueued.
 *   - Volumes are float32, layout vol[b][z][y][x] (x fastest), box edge N (even).  Voxel i on an
 *     axis sits at (i - N/2)/(N/2) in unit-ball coordinates; the ball is the set of voxels with
 *     (ix-N/2)^2 + (iy-N/2)^2 + (iz-N/2)^2 < (N/2)^2.
 *   - Coefficients are complex64 stored as interleaved float pairs (re, im), layout
 *     [b][l][k][m+l] for l = 0..Lmax, k = 0..K_l-1, m = -l..l; degree l starts at offsets[l]
 *     (bh_plan_layout).  They are the discrete inner product
 *     f_hat_klm = h^3 sum_{voxels in ball} f(x_v) conj(psi_klm(x_v)), h = 2/N, with
 *     c_lk = sqrt(2)/|j_{l+1}(lambda_lk)| (orthonormal psi) and complex Y_l^m with the
 *     Condon-Shortley phase.  Coefficients of real volumes satisfy
 *     f_hat_{k,l,-m} = (-1)^m conj(f_hat_klm); the matching calls rely on this symmetry.
 *   - Rotations are unit quaternions (w, x, y, z) in float32, the rotation by angle t about
 *     axis n being (cos t/2, sin t/2 n).  A rotation acts on volumes by (R f)(x) = f(R^{-1} x)
 *     and on coefficients by D^l_{mm'}(R) = <Y_l^m, R Y_l^m'>.  The score of R is
 *     <t, R f> = Re sum_l sum_{m,m'} xi^l_{mm'} D^l_{mm'}(R),  xi^l_{mm'} = sum_k conj(t_klm) f_klm'
 *     (Eq. 1 at s = 0 and Eq. 2).  When f = R_true t the maximiser is R_true^{-1}.
 *   - The gradient is taken along right perturbations R exp(eps J_i) about the body axes
 *     i = x, y, z.
 */
#ifndef BH_H
#define BH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define BH_OK 0
#define BH_PENDING 1          /* serving: the request is not finished yet */
#define BH_ERR_ARG (-1)       /* invalid argument (NULL pointer, size out of range, bad option) */
#define BH_ERR_CUDA (-2)      /* a CUDA runtime or driver call failed; the message names it */
#define BH_ERR_OOM (-3)       /* device or host allocation failed */
#define BH_ERR_BUDGET (-4)    /* serving: the request can never fit the HBM budget */
#define BH_ERR_TIMEOUT (-5)   /* a bounded device-side wait gave up; results are invalid */
#define BH_ERR_BUSY (-6)      /* serving: queue full, try again */
#define BH_ERR_UNSUPPORTED (-7) /* the device or configuration is not supported (not sm_103) */

/* marching schedules: at most BH_MAX_STAGES bands; a per-subtomogram schedule row (bh_align_opts.stage_table,
   bh_choose_bands) is a band count followed by the bands */
#define BH_MAX_STAGES 8
#define BH_STAGE_ROW (BH_MAX_STAGES + 1)

/* expansion arithmetic (bh_plan_opts.mode) */
#define BH_MODE_FP32 0        /* plain FP32 FFMA GEMM */
#define BH_MODE_BF16_SPLIT 1  /* tcgen05 BF16 tensor-core GEMM, hi/lo split: Xh*Th + Xh*Tl + Xl*Th, FP32 accum */

/* Thread-local message for the last failing call on this thread ("" if none). */
const char* bh_last_error(void);
/* Static name of a status code. */
const char* bh_status_string(int status);
/* Library ABI version (major * 10000 + minor * 100 + patch). */
int bh_version(void);

/* ------------------------------------------------------------------ host-only basis data */
/*
 * Radial data of the index set I = {(k,l,m): l <= Lmax, lambda_lk <= lambda_max} (Sec. II-A:
 * lambda_lk is the k-th positive root of j_l; c_lk the positive normalisation constant).
 * Computed in FP64 on the host; no GPU is touched.
 *   Lmax        0..64
 *   lambda_max  > 0; <= 0 is invalid here.  A root is kept when lambda_lk <= lambda_max + 1e-9.
 *   K           host, Lmax+1 ints: K[l] = number of roots kept for degree l.
 *   lambda, c   host, capacity `cap` doubles each, filled degree by degree (l = 0..Lmax, k ascending).
 * Returns BH_ERR_ARG if cap is smaller than sum_l K[l] (K is still filled).
 */
int bh_basis_roots(int Lmax, double lambda_max, int* K, double* lambda, double* c, int cap);

/* ------------------------------------------------------------------ plans */
typedef struct bh_plan bh_plan;

/* plan flags (bh_plan_opts.flags) */
#define BH_PLAN_MATCH_ONLY 1  /* no expansion table or scratch: the matching calls only (score, alignment,
                                 candidates, energy, re-scoring) on coefficients computed elsewhere */

typedef struct {
  int N;             /* box edge in voxels: even, 4..256 */
  int Lmax;          /* largest degree: 0..64 */
  double lambda_max; /* radial cutoff; <= 0 selects pi * N / 2 */
  int mode;          /* BH_MODE_FP32 or BH_MODE_BF16_SPLIT */
  int max_batch;     /* volumes per internal expansion pass (sizes the scratch); <= 0 selects 512 */
  int flags;         /* 0 or BH_PLAN_MATCH_ONLY */
} bh_plan_opts;

/*
 * Build a plan on the current CUDA device: roots and constants in FP64 on the host, the basis
 * table Psi[j][v] (real form, one row per coefficient slot, h^3 folded in) evaluated in FP64
 * and stored on the device in the arithmetic of `mode`, plus the expansion scratch.  With
 * flags = BH_PLAN_MATCH_ONLY the table and scratch are left out (64^3, l <= 32: 1.8 GB fewer in
 * BF16-split mode); the expansion calls and the shift search then fail with BH_ERR_ARG.
 * The plan owns all of its device memory and must be used with its device current (other
 * devices: BH_ERR_ARG).  Creation is synchronous.
 * Errors: BH_ERR_ARG (options), BH_ERR_OOM, BH_ERR_CUDA, BH_ERR_UNSUPPORTED (device is not
 * compute capability 10.3).
 */
int bh_plan_create(bh_plan** out, const bh_plan_opts* opts);
/* Free the plan (synchronises the device first).  NULL is accepted. */
int bh_plan_destroy(bh_plan* plan);
/*
 * Layout of the plan's coefficient vectors: *Nb = number of complex coefficients per volume,
 * *V = number of voxels inside the ball, offsets (host, Lmax+2 ints, may be NULL) with
 * offsets[l] = first slot of degree l and offsets[Lmax+1] = Nb.  Any output may be NULL.
 */
int bh_plan_layout(const bh_plan* plan, int* Nb, int* V, int* offsets);
/* Options the plan was created with (lambda_max resolved). */
int bh_plan_info(const bh_plan* plan, bh_plan_opts* opts);
/*
 * Shape of the plan's expansion GEMM.  Every real basis row is even or odd under each of the reflections
 * x -> -x, y -> -y, z -> -z, and the in-ball voxels are symmetric under them, so the expansion runs as 8
 * block products (one per parity class) over the fundamental voxels x, y, z >= 0 (octant folding, an exact
 * rewriting of the sum over voxels): *K = fundamental voxels padded to the K block, *N = table rows padded
 * class by class to the 128-row tile.  The multiply-adds per volume are K * N (against V * Nb unfolded).
 * Outputs may be NULL.
 */
int bh_plan_gemm(const bh_plan* plan, int* K, int* N);

/*
 * Error word of the plan's device waits.  Every wait of the tensor-core expansion pipeline (mbarrier
 * phases between the TMA producer, the MMA issuer and the epilogue) gives up after about 2 s of device
 * time, records the wait site and lets the kernel return, so a stalled pipeline never hangs the GPU.
 * bh_plan_status returns BH_ERR_TIMEOUT (and clears the word) if that happened since the last check,
 * else BH_OK; call it after synchronising the streams the plan's work ran on.  Synchronous.
 * bh_plan_probe_wait enqueues a probe in which one such wait runs out (a barrier phase that nothing
 * completes): about 2 s later bh_plan_status reports BH_ERR_TIMEOUT; the context stays usable.
 */
int bh_plan_status(bh_plan* plan);
int bh_plan_probe_wait(bh_plan* plan, void* stream);

/* ------------------------------------------------------------------ expansion */
/*
 * Expansion display of Sec. II-A on the voxel grid: coeffs[b] = f_hat of vols[b].
 *   vols    device, B * N^3 floats, layout [b][z][y][x].
 *   B       >= 0 (0 is a no-op).
 *   coeffs  device, B * Nb * 2 floats (complex interleaved), layout [b][l][k][m+l].
 * Uses the plan's scratch: calls on one plan must be serialised (same stream or synchronised).
 */
int bh_expand(bh_plan* plan, const float* vols, int B, float* coeffs, void* stream);

/*
 * Same result as bh_expand, for callers that cannot allocate device memory while they run -- for
 * example a thread recording into a stream that another component captures into a CUDA graph, or an
 * application that owns all device memory and only lends out pointers.  The paper has no counterpart:
 * this is a deployment variant of the expansion.
 *   Scratch: a fixed 64 MiB array compiled into the library (a file-scope __device__ array), held on
 *   every GPU where the library's module is loaded until the process exits.  The call allocates
 *   nothing (no cudaMalloc/cudaFree, no allocating library routine).
 *   Limit: one pass needs 128 * (8 K + N) * 4 bytes (K, N from bh_plan_gemm: the 8 parity-class
 *   projections of each volume over the fundamental voxels and the GEMM output); plans above 64 MiB
 *   per pass (for example N = 64, Lmax = 32: 88 MB) are rejected with BH_ERR_ARG.  Larger B is
 *   processed in several passes.
 *   Set-up: the first call on each device looks up the array's device address (cudaGetSymbolAddress)
 *   with that device current; make that first call before any stream capture.
 *   Sharing: all calls use the same array and it keeps the last call's contents (each pass overwrites
 *   what it reads, so nothing needs clearing); calls whose GPU work overlaps race on it.
 */
int bh_expand_noalloc(bh_plan* plan, const float* vols, int B, float* coeffs, void* stream);

/* ------------------------------------------------------------------ score and gradient */
/*
 * Eq. 2 at s = 0, truncated at band L, and its closed-form gradient (Sec. II-C) at given
 * rotations, one template against B subtomograms.
 *   tmpl    device, Nb complex: template coefficients t_hat.
 *   sub     device, B * Nb complex: subtomogram coefficients f_hat (real volumes).
 *   quats   device, B * S * 4 floats: rotations, [b][s][w,x,y,z]; normalised internally.
 *   S       1..512 rotations per subtomogram.
 *   L       band, 0..Lmax.
 *   score   device, B * S floats: Re sum_{l<=L} sum_{m,m'} xi^l_{mm'} D^l_{mm'}(R).
 *   grad    device, B * S * 3 floats or NULL: d score(R exp(eps J_i))/d eps at 0, i = x, y, z.
 */
int bh_score_grad(const bh_plan* plan, const float* tmpl, const float* sub, int B,
                  const float* quats, int S, int L, float* score, float* grad, void* stream);

/*
 * Energy of the cross-correlation coefficients per degree, E_l = sum_{m,m'} |xi^l_{mm'}|^2 for
 * l = 0..L (FP64 sums, stored as float).  The energy ratio of Fig. 1,
 * Ratio(L') = sum_{l>L'} E_l / sum_{l<=L} E_l (the caption's sum over m, m' made explicit), picks
 * high-energy bands for the marching schedule.
 *   tmpl        device, Nb complex (or n_templates * Nb with tmpl_index)
 *   sub         device, B * Nb complex
 *   tmpl_index  device, B ints or NULL
 *   energy      device, B * (L+1) floats, layout [b][l]
 */
int bh_energy(const bh_plan* plan, const float* tmpl, const float* sub, int B, int L, const int* tmpl_index,
              int n_templates, float* energy, void* stream);

/*
 * Marching bands chosen by the energy ratio (Fig. 1; Sec. II-C uses it to find high-energy bands and
 * Sec. III picks its L_set = {7, 12, 33} with it; the rule below is this library's reading), per
 * subtomogram: E_l = sum_{m,m'} |xi^l_{mm'}|^2 for l = 0..L (xi summed in FP32 over k, the energies in
 * FP64), Ratio(L') = sum_{l>L'} E_l / sum_{l<=L} E_l; band j is the smallest L' >= L_min with
 * Ratio(L') <= thresholds[j]; a band equal to the previous one is written once.  The rows feed
 * bh_align_batch (opts.stage_table) and bh_refine_fp64 without a round trip to the host.
 *   L             1..Lmax: the highest degree counted (and so the highest band a row can hold)
 *   tmpl_index, n_templates   as bh_align_opts (tmpl_index may be NULL)
 *   thresholds    host, n_thresholds doubles in (0, 1), strictly decreasing; n_thresholds 1..BH_MAX_STAGES
 *   L_min         1..L: the lowest band
 *   stage_table   device, B * BH_STAGE_ROW ints: row b = (number of bands, bands ascending)
 *   energy        device, B * (L+1) floats or NULL: E_l
 */
int bh_choose_bands(const bh_plan* plan, const float* tmpl, const float* sub, int B, int L, const int* tmpl_index,
                    int n_templates, const double* thresholds, int n_thresholds, int L_min, int* stage_table,
                    float* energy, void* stream);

/*
 * Score, gradient and Hessian of Eq. 2 (Newton steps, Sec. III) at S rotations per subtomogram, band L.
 * The Hessian is the second derivative of S(R exp(eps.J)) at eps = 0 (body frame, symmetric),
 * H_ij = -Re sum_l sum_{m,m'} xi^l_{mm'} [D^l(R) (J_i J_j + J_j J_i)/2]_{mm'}; it is evaluated through
 * Euler-angle derivatives and set to zero within sin(beta) <= 1e-4 of the Euler chart's poles.
 *   score  device, B * S floats;  grad  device, B * S * 3 floats or NULL
 *   hess   device, B * S * 6 floats (xx, xy, xz, yy, yz, zz) or NULL
 * Other arguments as bh_score_grad.
 */
int bh_score_hess(const bh_plan* plan, const float* tmpl, const float* sub, int B, const float* quats, int S,
                  int L, float* score, float* grad, float* hess, void* stream);

/* ------------------------------------------------------------------ alignment */
typedef struct {
  int group;              /* lanes cooperating on one start: 0 = autotuned, else 1, 2, 4, 8 or 16 */
  const int* tmpl_index;  /* device, B ints selecting a template row of `tmpl`, or NULL (row 0) */
  int n_templates;        /* rows in `tmpl` when tmpl_index is given */
  float* start_quat_out;  /* device, B * S * 4 floats or NULL: final rotation of every start */
  float* start_score_out; /* device, B * S floats or NULL: final score of every start */
  int starts_per_thread;  /* 0 = autotuned; 1, or 2 (S even: each thread advances two starts' recursions
                             through every orbit, sharing the table loads and coefficients) */
  int refine_fp64;        /* K in 0..64: after the FP32 ascent, re-score the K best starts (by FP32
                             score) at the last band with the d-recursion, seeds and phases in FP64
                             and the chain sums in compensated FP32 pairs (see bh_refine_fp64), and
                             select among them on that score (score_out then holds it, rounded to
                             float).  Needs start_quat_out and start_score_out.  0 = off */
  int newton;             /* 0: gradient ascent (Sec. II-C).  1: damped Newton steps (Sec. III): per
                             iteration, d = -H^{-1} g when -H is positive definite, else the gradient
                             step pi/(2L) g/|g|; d clipped to length pi/L and scaled by a damping factor
                             lam (1 at each stage start); the trial R exp(d.J) is accepted if it raises
                             the score (lam <- min(1, 2 lam)), else lam <- lam/2.  One start per thread
                             group (starts_per_thread 0 or 1); `group` may also be 32; 0 picks a
                             default (up to a warp per start when S is small and the band large) */
  const struct bh_wedge* wedge; /* NULL, or the missing-wedge norm from bh_wedge_create: maximise the
                             constrained score C(R) = S(R) / sqrt(Dn(R)), the common-region form of
                             Sec. II-B, with the ascent's step rule and marching instead of S(R); one
                             template (no tmpl_index), newton 0, starts_per_thread 0 or 1; score_out then
                             holds C.  Diagnostic, off by default: on voxel data with a missing wedge it
                             reproduces its FP64 reading but lands farther from the ground truth than the
                             plain score (1.8 against 1.0 degrees median on the 32^3 batch) */
  int dealing;            /* how a group's lanes share the orbits (m, n) of an evaluation: 0 = autotuned
                             (by rows when not tuned), 1 = row by row (lane q takes n = q - m + kG of row m),
                             2 = flat across rows (orbit m^2 + m + n to lane (m^2 + m + n) mod G; no lanes
                             idle at row ends; gradient ascent: group 4, 8 or 16, starts_per_thread 1 or
                             2; Newton steps: group 8, 16 or 32).  The constrained ascent (opts.wedge)
                             deals by rows and ignores it; results differ between dealings by FP32
                             rounding */
  const int* stage_table;  /* device, B * BH_STAGE_ROW ints or NULL: a marching schedule per subtomogram,
                             row b = (count, band_1 < band_2 < ...), e.g. from bh_choose_bands.  `stages`
                             then gives the largest band any row may use (shared memory, kernel variant)
                             and the schedule of rows whose count is 0; bands are clamped to
                             1..stages[nstages-1] and a band not above its predecessor is skipped.  With
                             refine_fp64 each subtomogram is re-scored at its own last band */
} bh_align_opts;


/*
 * Multi-start gradient ascent with frequency marching (Sec. II-C) for B subtomograms, in one
 * launch.  For every subtomogram and start: for each band L in `stages` (ascending, 1..Lmax):
 * h = pi/(2L), evaluate score and gradient, then `steps` times: stop if |g| <= 1e-12 |S|; else
 * u = g/|g|, trial R' = R exp(h u.J); accept if score(R') > score(R) (h <- min(1.5h, pi/L)),
 * else h <- h/2.  The result of a subtomogram is the start with the largest final score
 * (exact ties: lowest start index).
 *   tmpl       device, Nb complex (or n_templates * Nb with opts->tmpl_index).
 *   sub        device, B * Nb complex.
 *   starts     device, B * S * 4 floats: initial rotations.
 *   S          1..512 starts per subtomogram; S * group <= 512.
 *   stages     host, nstages ints (1..8 stages), strictly increasing, each in 1..Lmax.
 *   steps      ascent steps per stage, 0..100000.
 *   quat_out   device, B * 4 floats: best rotation R* (maximiser of <t, R f>).
 *   score_out  device, B floats: its score.
 *   opts       may be NULL (all defaults).
 */
int bh_align_batch(const bh_plan* plan, const float* tmpl, const float* sub, int B,
                   const float* starts, int S, const int* stages, int nstages, int steps,
                   float* quat_out, float* score_out, const bh_align_opts* opts, void* stream);

/*
 * The precision form's final refinement as a call of its own (bh_align_batch runs the same step when
 * opts->refine_fp64 = K): for every subtomogram, the K starts with the largest FP32 scores in
 * start_score (ties: lowest index) are scored at band L with the d-recursion, seeds and phases in FP64
 * (Eq. 2; the orbit table of P_l xi^l is rounded to FP32 once per entry).  Each orbit's sum over l of
 * recursion value times table entry is accumulated as an FP32 pair (the FP64 value split into two FP32
 * parts, products split exactly, error-free two-sums: within about 2^-43 of the sum of the terms'
 * magnitudes, against about 2^-48 for FP64 summation of a 33-term chain and 2^-24 for the table's own FP32
 * rounding), then combined with the phases in FP64.  The best of the K on that score is
 * written to quat_out / score_out (rounded to float) / score64_out.
 *   start_quat   device, B * S * 4 floats: final rotation of every start (opts->start_quat_out)
 *   start_score  device, B * S floats: their FP32 scores (opts->start_score_out)
 *   L            band, 0..Lmax;  K  1..min(64, S)
 *   tmpl_index   device, B ints or NULL (n_templates rows in tmpl), as in bh_align_opts
 *   stage_table  device, B * BH_STAGE_ROW ints or NULL (see bh_align_opts.stage_table): each subtomogram
 *                is then re-scored at the last band of its row (bands clamped to 1..L; L >= 1)
 *   score64_out  device, B doubles or NULL
 */
int bh_refine_fp64(const bh_plan* plan, const float* tmpl, const float* sub, int B, const float* start_quat,
                   const float* start_score, int S, int L, int K, const int* tmpl_index, int n_templates,
                   const int* stage_table, float* quat_out, float* score_out, double* score64_out, void* stream);

/* ------------------------------------------------------------------ shift search */
/*
 * Rotational matching over a grid of shifts (Eq. 1 over R^3 x SO(3); Sec. II-C: maximise Eq. 2 for a
 * shift s and repeat over a grid of shifts).  For every subtomogram f and integer-voxel shift s_j,
 * f_s(x) = f(x + s_j) (zero outside the box) is expanded, Eq. 2 with xi^s is maximised by the marching
 * ascent from the same starts, and the (shift, rotation) with the largest final score is returned.
 *   vols        device, B * N^3 floats
 *   shifts      host, nshift * 3 ints (sx, sy, sz) in voxels, each in (-N, N); nshift in 1..4096
 *   starts      device, B * S * 4 floats (used for every shift)
 *   workspace   device, >= bh_align_shifts_workspace(plan, B, nshift, S) bytes, 256-byte aligned
 *   shift_out   device, B ints: index j of the best shift
 *   quat_out    device, B * 4 floats; score_out device, B floats
 *   opts        as bh_align_batch (tmpl_index, group, starts_per_thread); per-start outputs and FP64
 *               re-scoring are not available here
 * Uses the plan's expansion scratch (serialise calls on one plan).
 */
size_t bh_align_shifts_workspace(const bh_plan* plan, int B, int nshift, int S);
int bh_align_shifts(bh_plan* plan, const float* tmpl, const float* vols, int B, const int* shifts, int nshift,
                    const float* starts, int S, const int* stages, int nstages, int steps, void* workspace,
                    size_t workspace_bytes, int* shift_out, float* quat_out, float* score_out,
                    const bh_align_opts* opts, void* stream);

/* ------------------------------------------------------------------ candidate starts */
/*
 * Rotation grid for candidate starts (Sec. III: the initial candidates are the local maxima of Eq. 2
 * truncated at the lowest selected band).  The grid is uploaded to the current device and its
 * neighbour lists are built there: j != i is a neighbour of i when |q_i . q_j| >= cos(radius / 2)
 * (geodesic angle <= radius), the dot product summed in the order w, x, y, z in FP64.
 *   quats   host, n * 4 floats (w, x, y, z), unit quaternions (|q|^2 within 1e-4 of 1, else
 *           BH_ERR_ARG); n in 1..16384; copied
 *   radius  neighbourhood radius in radians, [0, pi]
 * The grid is owned by the caller and freed by bh_grid_destroy.  Synchronous.
 */
typedef struct bh_grid bh_grid;
int bh_grid_create(bh_grid** out, const float* quats, int n, double radius);
int bh_grid_destroy(bh_grid* grid);
/* Grid size, largest neighbour count and total neighbour entries (any output may be NULL). */
int bh_grid_info(const bh_grid* grid, int* n, int* max_neighbors, long long* n_edges);
/* Copy the neighbour lists to the host in CSR form: offsets (n+1 ints), neighbors (cap >= n_edges ints,
   ascending within each list).  Synchronous. */
int bh_grid_neighbors(const bh_grid* grid, int* offsets, int* neighbors, long long cap);

/*
 * Candidate starts for B subtomograms.  For each subtomogram: Eq. 2 truncated at band L at every
 * grid rotation (FP32; the grid rotations are shared by all subtomograms, so their Wigner factors are
 * computed once per grid and band and the B x n scores are one dense contraction with the
 * subtomograms' orbit tables); grid point i ranks above j when its score is larger, or equal with
 * i < j; i is a local maximum when it ranks above all of its neighbours.  The candidates are the local
 * maxima in rank order followed, if there are fewer than S, by the other grid points in rank order;
 * the first S are written.  The first call for a band builds that band's factors for the grid
 * (synchronously, on a private stream); work memory (B x n scores) comes from stream-ordered
 * allocation on `stream`.
 *   L               band, 1..Lmax (the lowest marching band; one CTA's shared memory holds 8 bytes of
 *                   sort key per grid point -- per power of two above n when S > 64 -- at most 227 KB)
 *   tmpl, sub, tmpl_index, n_templates   as bh_align_batch
 *   S               1..n candidates per subtomogram
 *   starts_out      device, B * S * 4 floats: the candidate rotations (grid entries as given), ready
 *                   as `starts` of bh_align_batch
 *   index_out       device, B * S ints (grid indices) or NULL
 *   grid_score_out  device, B * n floats (band-L score of every grid rotation) or NULL
 */
int bh_candidates(const bh_plan* plan, const bh_grid* grid, const float* tmpl, const float* sub, int B, int L,
                  const int* tmpl_index, int n_templates, int S, float* starts_out, int* index_out,
                  float* grid_score_out, void* stream);

/* ------------------------------------------------------------------ missing wedge */
/*
 * Missing-wedge constrained correlation (Sec. II-B: correlate only where both volumes sample Fourier
 * space).  The subtomograms sample the directions |k_z| <= tan(a) |k_x| (tilt axis y, beam z, tilt
 * half-angle a); the template is complete.  Rotating a subtomogram by R rotates that region, so the
 * constrained score is C(R) = S(R) / sqrt(Dn(R)), Dn(R) = ||W_R t||^2, evaluated on the template's DFT
 * samples 0 < |k| < N/2 (plus k = 0) with the wedge indicator expanded in spherical harmonics up to
 * band L: Dn(R) = |T(0)|^2 + Re sum_{l<=L} sum_{m,m'} q_lm w_lm' D^l_{mm'}(R),
 * q_lm = sum_k Y_l^m(k/|k|) |T(k)|^2 (T: DFT of the template restricted to the ball), w_lm = <Y_l^m, W>.
 * bh_wedge_create prepares q and w on the host in FP64 (synchronous; about a second at 64^3) and keeps
 * them on the plan's device.
 *   tvol            host, N^3 floats: the template volume, layout [z][y][x]
 *   half_angle_deg  a in (0, 90)
 *   L               0..Lmax: the highest band the constrained alignment will use
 */
typedef struct bh_wedge bh_wedge;
int bh_wedge_create(const bh_plan* plan, const float* tvol, double half_angle_deg, int L, bh_wedge** out);
int bh_wedge_destroy(bh_wedge* wedge);
/* Host FP64 copies: q and w as (L+1)^2 complex values, interleaved (re, im), slot l^2 + m + l; |T(0)|^2. */
int bh_wedge_coeffs(const bh_wedge* wedge, double* q, double* w, double* c0);
/* Dn(R) and its body-frame gradient at S rotations (device quats S*4, dn S floats, grad S*3 floats or
   NULL), band L <= the wedge's. */
int bh_wedge_norm(const bh_plan* plan, const bh_wedge* wedge, const float* quats, int S, int L, float* dn,
                  float* grad, void* stream);

/* ------------------------------------------------------------------ autotuning */
typedef struct {
  int align_group;  /* lanes per start (per pair of starts when align_starts_per_thread = 2) chosen for
                       (band stages[nstages-1], S) */
  int align_starts_per_thread;
  float align_ms;   /* its time for B subtomograms */
  int gemm_bn;      /* N tile of the tensor-core expansion GEMM (BF16 mode; 0 in FP32 mode) */
  float expand_ms;  /* bh_expand time for B volumes with that tile */
  int align_dealing; /* orbit dealing of the chosen ascent variant (bh_align_opts.dealing) */
} bh_tune_result;

/*
 * Time the variants of the two hot kernels on synthetic data of this shape (B subtomograms, S starts,
 * the given marching schedule) and keep the fastest in the plan: bh_align_batch with group = 0 then
 * uses the chosen lanes-per-start for this (top band, S), and bh_expand the chosen GEMM N tile.
 * Allocates and frees its own temporary device buffers; synchronous.  `out` may be NULL.
 */
int bh_autotune(bh_plan* plan, int B, int S, const int* stages, int nstages, int steps, bh_tune_result* out);

/*
 * Time the Newton kernel (opts.newton) with 1, 2, 4, 8, 16 and 32 lanes per start dealt by rows and 8, 16
 * and 32 dealt in flat order for this shape, and keep the fastest in the plan for (band stages[nstages-1],
 * S); bh_align_batch with opts.newton and group 0 uses it.  out (may be NULL) receives align_group,
 * align_dealing and align_ms; align_starts_per_thread is 1, the other fields zero.  Synchronous; allocates
 * and frees its own scratch.
 */
int bh_autotune_newton(bh_plan* plan, int B, int S, const int* stages, int nstages, int steps, bh_tune_result* out);

/* ------------------------------------------------------------------ random starts */
/*
 * Uniform random rotations for the multi-start ascent (the paper starts from local maxima of the
 * lowest band instead; uniform starts are this library's default).  Host only.  Start s of
 * subtomogram b depends only on (seed, b, s): three uniforms from SplitMix64 at counters
 * seed + 3 (b S + s) + {0,1,2}, mapped by Shoemake's method to a unit quaternion with w >= 0.
 *   out  host, B * S * 4 floats, layout [b][s][w,x,y,z].
 */
int bh_random_starts(uint64_t seed, int B, int S, float* out);

/* ------------------------------------------------------------------ serving */
/*
 * A request loop with continuous batching: requests of uneven sizes and box edges arrive at any
 * time; a worker thread admits them while the HBM budget and a free stream slot allow, merges waiting
 * requests of the same box edge into one batch (expansion + one alignment launch with a
 * per-subtomogram template index), and keeps up to max_inflight bulk batches on the device at once on
 * separate streams.  Optionally, requests whose estimated device time is at most express_ms form an
 * express class with its own express_slots streams at the device's highest stream priority;
 * admission keeps arrival order within each class.  Batch
 * memory comes from the server's own stream-ordered pool, which keeps up to the budget mapped.  Where
 * the device reads pageable host memory coherently (cudaDevAttrPageableMemoryAccess, e.g. a Grace host
 * over NVLink-C2C), the expansion gathers each request's in-ball voxels straight from its host buffer:
 * no host->device copy of the volumes and no host thread blocked on one.
 * Template coefficients stay resident.  Each subtomogram's result
 * depends only on its own data, template, starts and the box's schedule -- not on what it was
 * batched with.  Schedule per box edge N: Lmax = N/2, lambda_max = pi N/2, bands Lmax/4, Lmax/2,
 * Lmax, `steps` ascent steps per band.
 */
typedef struct bh_server bh_server;

typedef struct {
  size_t hbm_budget_bytes; /* device bytes for in-flight batches (plans and templates excluded); 0 = 8 GiB */
  int max_inflight;        /* batches on the device at once (one stream each): 1..16; 0 = 4 */
  int max_batch;           /* subtomograms merged into one batch: 1..65536; 0 = 1024 */
  int queue_capacity;      /* requests waiting for admission; 0 = 65536 */
  int mode;                /* BH_MODE_* of the expansion for every box edge */
  int steps;               /* ascent steps per band; 0 = 30 */
  int newton;              /* 0: gradient ascent (Sec. II-C); 1: damped Newton steps (Sec. III; fewer steps
                              reach the same optimum, e.g. 8 per band) */
  int express_slots;       /* 0 (default): one class, every request bulk; 1..16: that many high-priority
                              streams for an express class of small requests */
  double express_ms;       /* estimated device time (ms) up to which a request, and a merged express
                              batch, is express; 0 = 2.0 */
  int ingest;              /* 0: read request volumes in place when the device reads pageable host memory
                              coherently, else copy them to the device; 1: always copy */
  int piece;               /* requests with more subtomograms are admitted in pieces of at most this many,
                              each next piece queued behind the requests that arrived meanwhile; results
                              do not depend on it (random starts are drawn per subtomogram); 0 = 128 */
} bh_serve_opts;

typedef struct {
  int template_id;     /* from bh_serve_add_template; fixes the box edge N */
  int B;               /* subtomograms, >= 1 */
  const float* vols;   /* host, B * N^3 floats [b][z][y][x]; must stay valid until the request completes */
  int S;               /* starts per subtomogram, 1..512 */
  const float* starts; /* host, B * S * 4 floats, or NULL: bh_random_starts(seed, B, S) */
  uint64_t seed;
  float* quat_out;     /* host, B * 4 floats, written before bh_serve_poll reports BH_OK */
  float* score_out;    /* host, B floats */
} bh_request;

typedef struct {
  uint64_t submitted, completed, batches;
  uint64_t express_batches; /* batches of the express class */
  uint64_t in_place_batches; /* batches whose volumes the expansion read in place from host memory */
  uint64_t queued;          /* waiting for admission */
  uint64_t inflight_batches;
  size_t inflight_bytes;    /* budget in use */
  uint64_t staging_allocs;  /* pinned staging (re)allocations, creation included */
  double launch_ms_total;   /* worker thread time spent enqueueing batches (copies, starts, launches) */
  double launch_ms_max;     /* longest single enqueue */
} bh_serve_counters;

/* Create a server on the current device.  Errors: BH_ERR_ARG, BH_ERR_CUDA, BH_ERR_UNSUPPORTED. */
int bh_serve_create(bh_server** out, const bh_serve_opts* opts);
/* Expand a template volume (host, N^3 floats) once and keep its coefficients resident; builds the
 * plan of box edge N on first use.  Synchronous.  *template_id receives its id. */
int bh_serve_add_template(bh_server* srv, int N, const float* vol, int* template_id);
/* Queue a request (non-blocking).  BH_ERR_BUDGET if its footprint alone exceeds the budget,
 * BH_ERR_BUSY if the queue is full, BH_ERR_ARG for malformed requests. */
int bh_serve_submit(bh_server* srv, const bh_request* req, uint64_t* ticket);
/* BH_OK once the request's outputs are written (latency_ms, may be NULL: submit to completion),
 * BH_PENDING before; BH_ERR_ARG for an unknown ticket; BH_ERR_CUDA if its batch failed. */
int bh_serve_poll(bh_server* srv, uint64_t ticket, double* latency_ms);
/* Like poll, blocking up to timeout_ms (< 0: forever); BH_ERR_TIMEOUT when the time runs out. */
int bh_serve_wait(bh_server* srv, uint64_t ticket, double timeout_ms, double* latency_ms);
/* Hold (1) or resume (0) admission of queued requests; work already admitted continues. */
int bh_serve_pause(bh_server* srv, int paused);
int bh_serve_stats(bh_server* srv, bh_serve_counters* out);
/* Finish admitted work, drop queued requests, free everything.  NULL is accepted. */
int bh_serve_destroy(bh_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* BH_H */
