/*
 * libgosma: C ABI of the GB300 (sm_103a) implementation of the GOSMA
 * branch-and-bound hot path (Campbell et al., "The Alignment of the
 * Spheres: Globally-Optimal Spherical Mixture Alignment for Camera Pose
 * Estimation").
 *
 * Conventions shared by every entry point
 *   - Plain pointers and sizes only.  Unless an argument says "device",
 *     pointers are host pointers; the library copies what it needs and the
 *     caller keeps ownership of every buffer it passes.
 *   - All floating-point inputs and outputs are IEEE double.
 *   - Return value: GOSMA_OK (0) or a negative GOSMA_E* code.  No C++
 *     exception crosses the ABI.  gosma_last_error() gives a message for the
 *     last failing call on a context.
 *   - A context is bound to one device and one CUDA stream; calls on one
 *     context must not run concurrently from several host threads.
 *   - Vectors are row-major: an array of n 3-vectors is n x 3 doubles.
 *   - Camera model (proof of Lemma 1): a camera with rotation R (world to
 *     camera) and centre t sees model point mu along R (mu - t)/|mu - t|.
 *     Rotations are angle-axis vectors r, R = R_r by Rodrigues' formula
 *     (Sec. 4.1).
 */
#ifndef GOSMA_H
#define GOSMA_H

#ifdef __cplusplus
extern "C" {
#endif

#define GOSMA_OK 0
#define GOSMA_EINVAL (-1)     /* invalid argument (sizes, weights, concentrations, ...) */
#define GOSMA_ENOMEM (-2)     /* device or host allocation failed */
#define GOSMA_ECUDA (-3)      /* a CUDA runtime call failed */
#define GOSMA_ETIMEOUT (-4)   /* a bounded device wait ran out */
#define GOSMA_ENOTREADY (-5)  /* mixtures or domain not set yet */

/* Result status of gosma_bnb_solve (gosma_result.status). */
#define GOSMA_OPTIMAL 0      /* d* - global lower bound <= eps (Algorithm 1 stopping rule) */
#define GOSMA_NODE_LIMIT 1   /* stopped at opts.max_nodes */
#define GOSMA_TIME_LIMIT 2   /* stopped at opts.max_seconds */
#define GOSMA_QUEUE_FULL 3   /* the device queue reached its capacity */
#define GOSMA_RUNNING 4      /* gosma_bnb_step returned before termination */

typedef struct gosma_ctx gosma_ctx;

/* A 6-orthotope C_r x C_t (Sec. 4.1): rotation cube with centre r0 and
 * half-width r_hw, translation cuboid with centre t0 and half-widths t_hw.
 * 80 bytes, the layout of 10 consecutive doubles. */
typedef struct {
    double r0[3];
    double r_hw;
    double t0[3];
    double t_hw[3];
} gosma_cube;

/* Per-cube bound record written by gosma_eval_bounds_detail (8 doubles). */
typedef struct {
    double lb;        /* Theorem 1 lower bound, = self_lb - 2 cross_ub          */
    double ub;        /* Theorem 1 upper bound f(R_r0, t0), +inf if t0 infeasible */
    double self_lb;   /* sum over i,j of the self-pair lower bounds             */
    double cross_ub;  /* sum over i,j of the cross-pair upper bounds            */
    double self_c;    /* self sum of f at the centre                            */
    double cross_c;   /* cross sum of f at the centre                           */
    double psi_r;     /* rotation uncertainty angle (Lemma 2)                   */
    double psi_t_max; /* max over model means of the translation angle (Lemma 3) */
} gosma_bound;

typedef struct {
    double eps;          /* tolerance on the normalised L2 distance f/C22 + 1 (Sec. 6 uses 0.1) */
    int pop;             /* hypercubes removed from the queue per iteration (Algorithm 1); each gives 8 children.
                            gosma_bnb_solve / _start: 0 = automatic, 2^23 / (n1 n2) clamped to [8192, 65536]
                            (8192 from 1024 pairs per cube up); gosma_bnb_solve_batch: per problem,
                            0 = automatic (the same rule for the largest mixture, clamped to
                            [64, 65536], at most capacity / 16 and 2^31 / (8 problems)), else
                            1..65536 with 8 x pop x problems < 2^31 */
    long long max_nodes; /* stop after this many evaluated sub-cubes (<= 0: no limit) */
    double max_seconds;  /* wall-clock limit (<= 0: no limit) */
    int use_sma;         /* run local refinement (SMA, Sec. 5) when a sub-cube improves d* */
    int sma_max_iter;    /* L-BFGS iterations per SMA call (<= 0: 100) */
    long long queue_capacity; /* device queue capacity in cubes (<= 0: library default) */
    int bound_block;     /* gosma_bnb_solve_batch: threads per block of the bound kernel, and */
    int bound_cubes;     /* sub-cubes per block (groups of bound_block / bound_cubes threads):
                            32x1, 32x2 (half-warp groups, for mixtures of at most 16 model
                            components), 64x1, 64x2, 128x1, 128x2, 128x4, 256x1, 256x2, 256x4,
                            512x1 or 1024x1; both 0 (the default): chosen by the autotuner.
                            The single-problem solver ignores them. */
} gosma_opts;

typedef struct {
    double R[9], r[3], t[3]; /* best pose (r canonical: |r| <= pi) */
    double objective;        /* d*: f at the best pose (FP64)      */
    double objective_norm;   /* d* divided by C22, plus 1          */
    double lower_bound;      /* global lower bound at termination   */
    double gap_norm;         /* (d* - lower_bound) / C22            */
    double c22;              /* C22 = 2 pi * integral of p2^2       */
    long long nodes;         /* sub-cubes evaluated                 */
    long long iterations;    /* Algorithm 1 loop iterations          */
    long long sma_calls;
    long long queue_peak;
    double seconds;
    int status;              /* GOSMA_OPTIMAL, GOSMA_NODE_LIMIT, ... */
    long long cross_pairs;   /* (cube, i, j) cross pairs bounded so far        */
    long long self_pairs;    /* (cube, i < m) self pairs bounded so far        */
    double bound_ms;         /* device time of the bound kernel (CUDA events)  */
    double iteration_ms;     /* device time of whole iterations (CUDA events)  */
    long long queue_size;    /* live sub-cubes in the queue                    */
    long long launches;      /* kernels the context has launched so far        */
    int block_size;          /* batched solver: threads per block of the bound kernel  */
    int cubes_per_block;     /* batched solver: sub-cubes per block of the bound kernel */
    int tunings;             /* batched solver: times the autotuner timed the shapes     */
    long long dstar_iteration; /* the iteration that last lowered d* (the final incumbent's) */
} gosma_result;

/* One independent alignment problem for gosma_bnb_solve_batch: the mixtures
 * (as in gosma_set_mixtures, host pointers, read during the call only) and
 * the translation domain (as in gosma_set_domain).  nclass > 1 makes it a
 * semantic problem with class sizes n1c, n2c and class weights w, as in
 * gosma_set_mixtures_classes; nclass <= 1 ignores those arrays. */
typedef struct {
    int n1;
    const double *mu1, *sigma1, *phi1;
    int n2;
    const double *mu2, *kappa2, *phi2;
    double t_lo[3], t_hi[3], zeta;
    int nclass;
    const int *n1c, *n2c;
    const double *w;
} gosma_problem;

/* Create a context on CUDA device `device`, issuing all work on `stream`
 * (a cudaStream_t; NULL means the legacy default stream).  The context owns
 * every device buffer it allocates.  Returns GOSMA_ECUDA when the device
 * cannot be used (no GPU, or a device that is not sm_103). */
int gosma_create(int device, void *stream, gosma_ctx **out);

/* Release the context and all its device memory.  NULL is accepted. */
void gosma_destroy(gosma_ctx *ctx);

/* Message for the last error on ctx ("" if none).  Valid until the next call. */
const char *gosma_last_error(const gosma_ctx *ctx);

/* Set the GMM theta_1 = {mu1 (n1 x 3), sigma1 (standard deviations), phi1}
 * and the vMFMM theta_2 = {mu2 (n2 x 3, unit vectors), kappa2, phi2}
 * (Sec. 4, Eq. GMM, Eq. vMFMM).  Deep-copies the arrays.  GOSMA_EINVAL when
 * n < 1, sigma <= 0, kappa <= 0, a weight < 0, |sum(phi) - 1| > 1e-9 or
 * ||mu2_j| - 1| > 1e-6. */
/* New mixtures or a new domain (gosma_set_mixtures, _classes, gosma_set_domain)
 * end a branch-and-bound run in progress: gosma_bnb_step, gosma_bnb_save and
 * gosma_bnb_set_incumbent then return GOSMA_ENOTREADY until the next
 * gosma_bnb_start or gosma_bnb_load; gosma_bnb_history still reads the
 * ended run. */
int gosma_set_mixtures(gosma_ctx *ctx, int n1, const double *mu1, const double *sigma1, const double *phi1, int n2,
                       const double *mu2, const double *kappa2, const double *phi2);

/* Semantic form (Sec. 4.2): f = sum_l w_l f_l over nclass classes, f_l the
 * objective of Lemma 1 between class l's model and image mixtures.  The
 * components are given class by class: the first n1c[0] model and n2c[0]
 * image components belong to class 0, and so on; each class's weights phi1
 * and phi2 sum to 1; w_l >= 0 (the paper uses 1 / nclass).  Pairs interact
 * only within a class; ε applies to f / C22 + 1 with C22 = sum_l w_l C22_l.
 * The translation domain excludes the points within zeta of any class's
 * means.  Validation as in gosma_set_mixtures, per class; GOSMA_EINVAL for
 * an empty class. */
int gosma_set_mixtures_classes(gosma_ctx *ctx, int nclass, const int *n1c, const int *n2c, const double *w,
                               const double *mu1, const double *sigma1, const double *phi1, const double *mu2,
                               const double *kappa2, const double *phi2);

/* Rotation uncertainty angle of Lemma 2 used in the cross pairs of every
 * bound the context computes afterwards (gosma_eval_bounds, the
 * branch-and-bound solvers).  The paper gives the angle as a maximum over
 * the rotation cube's surface without a closed form; both modes bound it:
 *   GOSMA_PSI_R_CUBE (default): sqrt(3) h (capped at pi), the same for
 *     every direction, from angle(R_r p, R_r0 p) <= |r - r0|;
 *   GOSMA_PSI_R_POINT: one angle per model direction p = v_i (at the
 *     cuboid centre): sin(psi / 2) <= max over the cube's vertices d of
 *     |J_r(r0) d / 2 x p| + 3 h^2 / 8 (J_r the right Jacobian of the
 *     exponential map of SO(3)), never above the GOSMA_PSI_R_CUBE angle.
 * It is 13% smaller on average for small cubes and costs O(n1) per cube,
 * nothing per pair.  Branching (Sec. 4.1) keeps comparing the
 * point-independent angle, and gosma_bound.psi_r reports it.  GOSMA_EINVAL
 * for another mode. */
#define GOSMA_PSI_R_CUBE 0
#define GOSMA_PSI_R_POINT 1
int gosma_set_psi_r_mode(gosma_ctx *ctx, int mode);

/* Translation domain Omega_t: the cuboid [t_lo, t_hi] minus the points
 * within zeta of any model mean (Sec. 4.1).  zeta >= 0, t_lo < t_hi. */
int gosma_set_domain(gosma_ctx *ctx, const double t_lo[3], const double t_hi[3], double zeta);

/* Theorem 1 bounds for n cubes: lb[k] <= min of f over the feasible part of
 * cube k, ub[k] = f at its centre (+inf when the centre is within zeta of a
 * mean).  Cubes with no feasible pose (rotation part outside the pi-ball,
 * translation part within zeta of one mean) get lb = ub = +inf.
 * Pair terms are computed in FP32 (log domain) with a rounding slack that
 * keeps lb at or below the exact-arithmetic bound; per-cube sums are FP64.
 * on_device = 0: cubes, lb, ub are host pointers; the call returns when the
 * results are in place.  Where the device can address ordinary host memory
 * through the host page tables (a coherent CPU-GPU link), the kernels read
 * and write these arrays in place; otherwise they are staged through pinned
 * buffers in pipelined chunks (environment GOSMA_STAGED_HOST_IO=1 at
 * gosma_create forces the staged path).
 * on_device = 1: they are device pointers on the context's device; the call
 * is then asynchronous on the context's stream.  n = 0 is a no-op. */
int gosma_eval_bounds(gosma_ctx *ctx, const gosma_cube *cubes, int n, double *lb, double *ub, int on_device);

/* Same bounds, with the full per-cube record (gosma_bound, 8 doubles). */
int gosma_eval_bounds_detail(gosma_ctx *ctx, const gosma_cube *cubes, int n, gosma_bound *out, int on_device);

/* f(R_r, t) of Lemma 1 in FP64 on the device (host pointers). */
int gosma_eval_objective(gosma_ctx *ctx, const double r[3], const double t[3], double *f);

/* f and its gradient with respect to (r, t) in FP64 on the device, for
 * `count` poses x (count x 6: r then t, host pointers); any count >= 0
 * (the poses are processed in launches of at most 65,535). */
int gosma_eval_objective_grad(gosma_ctx *ctx, int count, const double *x, double *f, double *grad);

/* Allocation-free variant of gosma_eval_objective_grad (the paper has no
 * counterpart; it exists for callers that cannot let the library allocate
 * device memory while they run: real-time loops that size all memory at
 * start-up and cannot afford cudaMalloc's implicit device synchronisation,
 * and applications that own the device-memory budget themselves).
 * d_x: device pointer, count x 6 doubles (r then t per pose).
 * d_out: device pointer, count x 7 doubles (f, df/dr (3), df/dt (3) per pose).
 * Both stay owned by the caller.  The kernels run asynchronously on the
 * context's stream; no host copy, no synchronisation, no allocation.
 * Scratch lives in one fixed 8 MiB device array inside the library, held by
 * every GPU that loads it until the process exits: the call returns
 * GOSMA_EINVAL when count * (128 n1 + 56 ceil((n1^2 + n1 n2) / 512)) bytes
 * exceeds it.  All calls on a device share that array, so calls whose kernels
 * overlap on the GPU (e.g. issued on different streams) race.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  The address is kept for
 * the life of the process, so do not cudaDeviceReset a device between calls.
 * (The size limit also keeps count below 65,536, the kernels' grid limit.) */
int gosma_eval_objective_grad_noalloc(gosma_ctx *ctx, int count, const double *d_x, double *d_out);

/* SMA (Sec. 5) from `count` seed poses at once, on the device: each seed is
 * refined by L-BFGS (memory 8, backtracking Armijo line search, first step
 * 0.01 in the largest coordinate) on f of Lemma 1, restricted to feasible
 * poses (translation inside the domain of gosma_set_domain and at least zeta
 * from every model mean; infeasible trial poses halve the step unevaluated).
 * A thread block runs a seed's whole refinement with no host round trip.
 * x0: count x 6 seeds (r then t).  max_iter >= 0: L-BFGS iterations per seed
 * (0 returns the seeds with their f).
 * precision 64: f and its gradient in FP64 throughout.  precision 32: the
 * search evaluates them in FP32 and also stops once an iteration gains less
 * than 2^-26 times the sum of the terms' magnitudes or 20 halvings of the
 * step find no decrease; the returned f is still FP64.
 * Outputs: x (count x 6, may alias x0) the refined poses; f (count) the FP64
 * objective at x, +inf for an infeasible seed (whose x is the seed).  f is
 * evaluated in FP64 at the refined pose and at the seed, and the better of
 * the two is returned, so f never exceeds the seed's f; grad
 * (count x 6 or NULL) the FP64 gradient at x (0 for infeasible seeds); iters
 * (count or NULL) the accepted iterations per seed, -1 for infeasible seeds.
 * on_device = 0: host pointers, the call returns with the results in place.
 * on_device = 1: device pointers on the context's device; asynchronous on
 * the context's stream.  Requires gosma_set_mixtures and gosma_set_domain
 * (GOSMA_ENOTREADY otherwise); GOSMA_EINVAL for count < 0, max_iter < 0,
 * another precision, null seeds or outputs, or mixtures whose FP32 tables
 * (36 n1 + 24 n2 bytes) exceed one block's shared memory. */
int gosma_sma_batch(gosma_ctx *ctx, int count, const double *x0, int max_iter, int precision, double *x, double *f,
                    double *grad, int *iters, int on_device);

/* Mixture generation (Sec. 6): the model's point set is clustered with
 * DP-means and a maximum-likelihood GMM is fitted to the clusters, the
 * theta_1 of gosma_set_mixtures.  One pass visits the points in index order;
 * a point whose squared distance to every current centre exceeds lambda
 * opens a new cluster centred on itself (seen by the later points of the
 * pass), every other point joins its nearest centre (lowest index on ties);
 * after the pass each centre becomes its cluster's mean and empty clusters
 * are removed, the others keeping their order.  Start: one cluster at the
 * mean of all points; stop: a pass that changes no label, or max_iter
 * passes.  Coordinates are first rounded to multiples of 2^-32 (of the
 * input's unit), which makes every cluster sum exact; the result is
 * deterministic and equals a serial double-precision run of the same steps.
 * Fit: phi_k = n_k / n, mu_k the mean, sigma_k = sqrt(sum |x - mu_k|^2 /
 * (3 n_k)) floored at sigma_min.
 * x: n x 3 host array, 1 <= n <= 2^26, n * max|x| < 2^30.  lambda > 0 (squared
 * distance), max_iter >= 1, 1 <= kmax <= 8192, sigma_min > 0.
 * Outputs (host): *k clusters; mu (kmax x 3), sigma (kmax), phi (kmax), of
 * which the first *k entries are written; labels (n, or NULL) the cluster of
 * every point; passes (or NULL) the passes run.  GOSMA_EINVAL (with *k = -1)
 * when more than kmax clusters would be needed. */
int gosma_dp_means(gosma_ctx *ctx, int n, const double *x, double lambda, int max_iter, int kmax, double sigma_min,
                   int *k, double *mu, double *sigma, double *phi, int *labels, int *passes);

/* Mixture generation (Sec. 6) for the image: the bearing vectors (n x 3,
 * unit length within 1e-6, n < 2^22) are clustered with DP-vMF-means, the
 * same passes as gosma_dp_means with the cosine x . mu as the similarity: a
 * vector whose cosine with every centre is below lambda opens a cluster, the
 * others join the most similar centre, and a centre is the normalised sum of
 * its members (its lowest-index member if that sum is exactly zero).
 * Coordinates are rounded to multiples of 2^-40 first.  Fit: phi_k = n_k /
 * n, mu_k the mean direction, kappa_k the maximum-likelihood concentration
 * on S^2, solving coth(kappa) - 1/kappa = |sum x| / n_k, capped at kappa_max
 * (> 1e-12).  The theta_2 of gosma_set_mixtures.  Arguments and errors as in
 * gosma_dp_means. */
int gosma_dp_vmf_means(gosma_ctx *ctx, int n, const double *x, double lambda, int max_iter, int kmax,
                       double kappa_max, int *k, double *mu, double *kappa, double *phi, int *labels, int *passes);

/* Algorithm 1 (GOSMA) on the device: branch, bound, prune and select run in
 * device kernels; d* is always an FP64 evaluation of f, refined by SMA
 * (Sec. 5) whenever a sub-cube's upper bound beats it.  opts may be NULL
 * (eps = 0.1, automatic pop, no limits, SMA on).  Equivalent to
 * gosma_bnb_start followed by gosma_bnb_step(ctx, 0, out). */
int gosma_bnb_solve(gosma_ctx *ctx, const gosma_opts *opts, gosma_result *out);

/* Algorithm 1 for nprob (<= 65535) independent problems at once, each with
 * its own mixtures, domain and queue segment.  Every iteration pops the
 * opts->pop best hypercubes (exact radix select on the FP32 lower-bound key,
 * ties in queue order) from each unfinished problem, bounds the children of
 * all problems in one persistent kernel launch, and replaces each problem's
 * d* by the exact FP64 objective at its best child's centre when smaller.
 * Every 8 iterations the host refines each problem whose d* improved with
 * L-BFGS (SMA, Sec. 5) in lock step, all such problems' poses in one FP64
 * launch per step (opts->use_sma, opts->sma_max_iter).  The iteration runs
 * as a captured CUDA graph on a private stream.  The bound kernel's shape
 * (threads per block, sub-cubes per block) is the caller's
 * (opts->bound_block, opts->bound_cubes) or picked by an autotuner: each
 * candidate shape is launched once and then timed three times on the same
 * sample of children (every few runs of four siblings, across all problems:
 * a sixteenth of the iteration, at least 64 children per SM) at
 * the fifth iteration; the smallest median wins if it is at least 3% below
 * the default shape's (128 threads, one sub-cube), and a winner by less
 * than 15% must also beat it in a full launch on the same children, else
 * the default stays; the shapes
 * are timed again (and the graph captured anew) whenever the number of
 * unfinished problems has halved since the last tuning, at least 32
 * iterations after it; results[k] reports
 * the final shape and the number of tunings.  The bounds of one sub-cube
 * differ between shapes only by the order of their FP32 sums.
 * results[k].seconds is the device time from the start to problem k's
 * certificate.  opts->queue_capacity is per problem (default 2^18
 * sub-cubes; two buffers of that size are allocated per problem),
 * opts->max_nodes per problem.  opts may be NULL (eps = 0.1, automatic pop, SMA
 * on).  Problems with invalid data make the call fail with GOSMA_EINVAL
 * before any work. */
int gosma_bnb_solve_batch(gosma_ctx *ctx, int nprob, const gosma_problem *probs, const gosma_opts *opts,
                          gosma_result *results);

/* Options of the learned form of the batched solver (an extension of the
 * method, not in the paper).  With use_mlp set (parameters loaded by
 * gosma_mlp_set_params), the queue-ordering network scores every child on
 * the tensor cores inside the iteration:
 *   - ordering: a child's pop priority is lb - beta * C22 * sigmoid(logit);
 *     the lower bound, pruning and the stopping test still use lb alone, so
 *     the certificate is the plain method's;
 *   - seeding (seed != 0): the best-scored child of each problem proposes a
 *     pose (its centre plus the predicted offset times its half-widths,
 *     clamped to the cube) whose exact FP64 objective competes for d* and is
 *     then refined by SMA.
 * trace_cap > 0 records up to trace_cap popped sub-cubes per problem. */
typedef struct {
    int use_mlp;
    float beta;
    int seed;
    int trace_cap;
    int active_iters;  /* score only during the first active_iters iterations (0: always) */
} gosma_learn_opts;

/* One popped sub-cube of a trace: the network's 16 input features as the
 * device computed them at pop time, the cube (r0, r half-width, t0,
 * t half-widths), its bounds and the incumbent at that time. */
typedef struct {
    float feat[16];
    double cube[10];
    double lb, ub, dstar;
    int problem, iteration;
} gosma_trace_rec;

/* gosma_bnb_solve_batch with the learned form and tracing.  lopts may be
 * NULL (plain).  trace (host, nprob * lopts->trace_cap records) and
 * trace_count (host, nprob) receive each problem's records in pop order
 * when lopts->trace_cap > 0.  GOSMA_ENOTREADY if use_mlp is set without
 * parameters. */
int gosma_bnb_solve_batch_ex(gosma_ctx *ctx, int nprob, const gosma_problem *probs, const gosma_opts *opts,
                             const gosma_learn_opts *lopts, gosma_result *results, gosma_trace_rec *trace,
                             int *trace_count);

/* Start a branch-and-bound run (the queue holds the root Omega_r x Omega_t).
 * The run's device state belongs to the context until the next start. */
int gosma_bnb_start(gosma_ctx *ctx, const gosma_opts *opts);

/* Run at most max_iters iterations of Algorithm 1 (max_iters <= 0: until a
 * stopping rule fires) and report the state in out (status GOSMA_RUNNING
 * while none has).  GOSMA_ENOTREADY without a prior gosma_bnb_start. */
int gosma_bnb_step(gosma_ctx *ctx, int max_iters, gosma_result *out);

/* ---------------------------------------------------------------------
 * Queue-ordering network (an extension of the method, not in the paper): a
 * 16 -> 128 -> 128 -> 16 MLP with GELU (exact erf form) whose output 0 is a
 * priority logit for a sub-cube and outputs 1..6 a seed-pose offset from the
 * cube centre in half-width units.  Weights and activations are BF16 on the
 * tensor cores with FP32 accumulation; an FP32 master copy of the
 * parameters is kept for training.  Packed parameter layout (FP32,
 * GOSMA_MLP_NPARAM values): W1 [128 x 16], b1 [128], W2 [128 x 128],
 * b2 [128], W3 [16 x 128], b3 [16], matrices row-major [out x in].
 * --------------------------------------------------------------------- */
#define GOSMA_MLP_NPARAM 20752

/* Load parameters (host array, copied) and reset the optimiser state. */
int gosma_mlp_set_params(gosma_ctx *ctx, const float *params);

/* Copy the FP32 master parameters to the host.  GOSMA_ENOTREADY before
 * gosma_mlp_set_params. */
int gosma_mlp_get_params(gosma_ctx *ctx, float *params);

/* Forward pass: x (n x 16, host) -> y (n x 16, host), FP32. */
int gosma_mlp_forward(gosma_ctx *ctx, int n, const float *x, float *y);

/* Parameter gradient (packed layout, host) of sum_rows dy . y(x) for an
 * upstream gradient dy (n x 16, host); dy is rounded to BF16 as in training. */
int gosma_mlp_grad(gosma_ctx *ctx, int n, const float *x, const float *dy, float *grad);

/* `steps` Adam steps (lr, betas 0.9 / 0.999) on minibatches of `batch` rows
 * (a multiple of 128; n a multiple of batch) taken in order, cyclically, from
 * the device-resident data set x (n x 16), label (n, in [0, 1]) and target
 * (n x 6).  Loss per row: logistic loss of y[0] against label plus
 * lam * label * |y[1..6] - target|^2.  losses (host, steps values, may be
 * NULL) receives the mean loss of each minibatch before its step. */
int gosma_mlp_train(gosma_ctx *ctx, int n, const float *x, const float *label, const float *target, int batch,
                    int steps, float lr, float lam, float *losses);

/* One iteration of a run (the quantities of Fig. 5): iteration number,
 * seconds since the start, d*, the global lower bound, live sub-cubes and
 * nodes so far. */
typedef struct {
    long long iteration;
    double seconds, dstar, lower_bound;
    long long queue_size, nodes;
} gosma_trace_point;

/* The per-iteration history of the current (or last) run of
 * gosma_bnb_start / gosma_bnb_step / gosma_bnb_solve: *count receives the
 * number of iterations, and the first min(count, max_points) points are
 * copied to out (max_points = 0: count only).  A resumed run starts a new
 * history. */
int gosma_bnb_history(gosma_ctx *ctx, long long max_points, gosma_trace_point *out, long long *count);

/* Offer an incumbent found elsewhere to the run in progress (between
 * gosma_bnb_step calls): another shard of the same problem, or a caller's own
 * refinement.  x: the pose (r then t, 6 doubles), f its objective value, which
 * the caller guarantees (the run does not re-evaluate it).  When f < d*, d*
 * and the best pose become (f, x): the next iterations prune against f and
 * Algorithm 1's stopping test uses it; otherwise nothing changes.  Used by
 * the sharded solve across GPUs, where every rank searches a slab of the
 * translation domain and the ranks exchange (d*, lower bound) between steps.
 * GOSMA_ENOTREADY without a run in progress, GOSMA_EINVAL for a NaN f or a
 * null x. */
int gosma_bnb_set_incumbent(gosma_ctx *ctx, double f, const double x[6]);

/* The children bounded by the last iteration of the run (Algorithm 1, "evaluate
 * the bounds of the sub-cubes"), in child order (parent k gives children
 * 8k .. 8k+7), as the bound kernel wrote them: cubes[c] the child's sub-cube
 * (decoded from its cell), bounds[c] its record as in gosma_eval_bounds_detail,
 * where lb, ub, self_lb, self_c and psi_t_max are the values the solver uses
 * (self_lb and self_c of a child of a rotation split are its parent's cached
 * sums), psi_r is Lemma 2's angle of the child's rotation cube, and cross_ub and
 * cross_c are derived from them (lb = self_lb - 2 cross_ub - 1e-12 (self_lb + 2
 * cross_ub), ub = self_c - 2 cross_c).  Infeasible children have every field
 * +inf but the angles.  *count receives the number of children (0 before the
 * first iteration); the first min(count, max_children) are copied (host
 * arrays).  Read-only: the run continues unchanged.  GOSMA_ENOTREADY without a
 * run. */
int gosma_bnb_last_children(gosma_ctx *ctx, int max_children, gosma_cube *cubes, gosma_bound *bounds, int *count);

/* A queue record of a branch-and-bound run (64 bytes): a sub-cube as cell
 * coordinates of the run's domain (rotation cube r at level lr of the
 * circumscribing cube [-pi, pi]^3, translation cuboid t at level lt of the
 * domain), its Theorem 1 lower bound and the self sums of its cuboid.  Only
 * meaningful to runs of the same mixtures and domain. */
typedef struct {
    double lb;                /* lower bound of f over the sub-cube           */
    double self_lb, self_c;   /* self sums of the cuboid (valid when flags & 1) */
    unsigned int r[3], t[3];  /* cell coordinates                              */
    unsigned short lr, lt;    /* levels (halvings) of the rotation and translation parts */
    float psit;               /* largest psi_t over the cuboid (split rule)   */
    unsigned int flags;
    float ubf;                /* upper bound at the centre (FP32), when known */
} gosma_node;

/* Move sub-cubes between runs of one problem (Algorithm 1 over several
 * solvers: their queues together hold the live sub-cubes, so the global
 * lower bound is the smallest of the runs' lower bounds).  Between
 * gosma_bnb_step calls:
 *   gosma_bnb_export drops the queued sub-cubes whose lower bound is not
 *   below d*, then removes up to max_nodes of the others (the most recently
 *   queued) from the run and writes them to out (host, max_nodes records);
 *   *count receives how many.  The run's lower bound is recomputed.
 *   gosma_bnb_import appends n records (host) to the run's queue (a run that
 *   had certified, with an empty queue, runs again); GOSMA_EINVAL when a
 *   record is not one of this library's or the queue would overflow.
 * Both: GOSMA_ENOTREADY without a run in progress.  The records must come
 * from a run of the same mixtures and domain. */
int gosma_bnb_export(gosma_ctx *ctx, int max_nodes, gosma_node *out, int *count);
int gosma_bnb_import(gosma_ctx *ctx, int n, const gosma_node *in);

/* Checkpoint of a run between two gosma_bnb_step calls: the solver record,
 * the incumbent and its pose, and every queue slot (keys and sub-cubes) go
 * to the file at path.  GOSMA_ENOTREADY without a run. */
int gosma_bnb_save(gosma_ctx *ctx, const char *path);

/* Resume a checkpoint on a context holding the same mixtures and domain
 * (GOSMA_EINVAL otherwise): later gosma_bnb_step calls continue the run
 * exactly as the saved one would have continued.  "Same mixtures" is
 * checked on the sizes, C22 and a 64-bit fingerprint of every mixture array
 * (means, scales, concentrations, class-weighted weights, classes), so a
 * file from another problem of the same sizes is refused. */
int gosma_bnb_load(gosma_ctx *ctx, const char *path);

/* Number of kernels the context has launched since it was created. */
long long gosma_kernel_launches(const gosma_ctx *ctx);

/* Failure detection without a fault: a kernel waits, with the time limit
 * the tensor-core kernels use (here limit_seconds, 0 < limit <= 10), on an
 * mbarrier that nothing arrives on.  The wait gives up and the call returns
 * GOSMA_ETIMEOUT; the context stays usable. */
int gosma_selftest_wait_timeout(gosma_ctx *ctx, double limit_seconds);

/* Testing of error paths: the next n device allocations of this context
 * fail as if the device were out of memory (the calls that needed them
 * return GOSMA_ECUDA and leave the context usable).  n = 0 turns it off. */
int gosma_debug_fail_allocations(gosma_ctx *ctx, int n);

/* Diagnostics: measured maximum relative error of the device's approximate
 * ex2, lg2, rcp, rsqrt and sqrt against FP64 over dense samples (5 values,
 * in that order), and the error bounds the bound kernel's slack assumes. */
int gosma_selftest_approx(gosma_ctx *ctx, double measured[5], double assumed[5]);

/* Diagnostics (no counterpart in the paper): measured throughput of the
 * pipes the bound kernel runs on, in lane operations per SM per clock cycle
 * at the device's maximum SM clock (*clock_mhz receives it): rates[0] scalar
 * FP32 fused multiply-add, rates[1] packed FP32x2 fused multiply-add (lanes,
 * two per instruction), rates[2] ex2.approx, rates[3] sqrt.approx, rates[4]
 * rcp.approx, rates[5] rsqrt.approx, rates[6] lg2.approx (each rcp and lg2
 * beside one FP32 add).  Each is timed with CUDA events over one launch of 8 x 256
 * threads per SM running eight independent chains of that instruction (best
 * of three launches after a warm-up).  A few milliseconds of device time. */
int gosma_selftest_pipe_rates(gosma_ctx *ctx, double rates[7], double *clock_mhz);

/* Diagnostics: the rotation matrices R_r of Rodrigues' formula (Sec. 4.1)
 * as the bound kernels' pre-pass forms them (double-float arithmetic, each
 * entry an unevaluated sum of two floats, returned as their FP64 sum), for
 * n >= 0 rotation vectors r (host, n x 3); R (host, n x 9, row-major per
 * vector) receives them.  For checking their accuracy against an FP64
 * rotation; n = 0 is a no-op. */
int gosma_selftest_rodrigues(gosma_ctx *ctx, int n, const double *r, double *R);

#ifdef __cplusplus
}
#endif
#endif /* GOSMA_H */
