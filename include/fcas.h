/*
 * fcas.h -- C ABI of the GB300 coherent-fitness library (libfcas.so).
 *
 * The library evaluates the network GLRT coherent fitness of a fully-coherent all-sky search for
 * compact-binary inspirals (Normandin & Mohanty, arXiv:2002.02150):
 *
 *   Gamma^2(Theta) = max over (t_c, A_1..A_4) of 2 lambda^(D),   Theta = (alpha, delta, tau0, tau1.5)
 *
 * (Sec. II.C, eq. gammaSqd, with the log-likelihood ratio of eq. loglikelihood and the inner
 * product of eq. innprod), organised as in Sec. II.D: over-whitened data, precomputed template
 * norms and the arrival delay moved onto the data (eq. data_template_innprod). The factor 2 makes
 * a noiseless injection at the true parameters return its network SNR^2 (eq. optimalSNR).
 *
 * Conventions shared by every entry point
 *  - Return value: FCAS_OK (0) on success, a negative FCAS_ERR_* code otherwise; the message of
 *    the last failure on the calling thread is returned by fcas_last_error().
 *  - Pointers marked "host or device" may point to host memory or to CUDA device memory; the
 *    library tells them apart with cudaPointerGetAttributes. When every pointer argument of a
 *    call is a device pointer the call is asynchronous on `stream`; when any is a host pointer the
 *    call returns only after the results have been copied into it.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - The caller keeps ownership of every buffer it passes; the context owns everything it
 *    allocates. A context must not be used from two threads at once.
 *  - A context belongs to the CUDA device that was current when it was created: every call that
 *    takes it must be made with that device current (FCAS_ERR_INVALID otherwise).
 *  - All floating-point inputs are IEEE binary64.
 */
#ifndef FCAS_H
#define FCAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FCAS_MAX_DET 8

enum fcas_status {
    FCAS_OK = 0,
    FCAS_ERR_INVALID = -1,   /* bad size, NULL pointer, non-finite or out-of-range input */
    FCAS_ERR_NOMEM = -2,     /* a device or host allocation failed */
    FCAS_ERR_CUDA = -3,      /* a CUDA runtime call or kernel launch failed */
    FCAS_ERR_TIMEOUT = -4,   /* a bounded device-side wait gave up (reserved) */
    FCAS_ERR_STATE = -5      /* the context is not in a state that allows the call */
};

enum fcas_precision {
    FCAS_PREC_FP64 = 0,      /* plain form: phase, products, FFTs and projection in binary64 */
    FCAS_PREC_FP32 = 1,      /* FP32 products/FFTs/projection; chirp and delay phase as
                                float-float (hi + lo) values reduced mod 1 turn (the delay
                                phasors' per-particle step in binary64; adjacent bins' chirp
                                phase stepped from a shared bin where the step's error is
                                below 1e-7 turns) */
    FCAS_PREC_FF = 2         /* binary64-class accuracy on the FP32 units: phase and detector sums
                                in binary64, transforms and projection in float-float (double-word)
                                arithmetic; spectrum, tables and intermediate as in the binary64 form */
};

/* One interferometer: ECEF position and unit vectors along its two arms (Sec. II, eq. detresponse:
 * the detector tensor is d = (x x^T - y y^T) / 2). */
typedef struct fcas_detector {
    double r[3];      /* ECEF position [m] */
    double xarm[3];   /* unit vector along the x arm */
    double yarm[3];   /* unit vector along the y arm */
} fcas_detector;

/* Data segment description. */
typedef struct fcas_setup {
    int32_t n_det;       /* D, 1..FCAS_MAX_DET */
    int32_t precision;   /* enum fcas_precision */
    int64_t n_samples;   /* samples per detector actually present, 1..n_fft */
    int64_t n_fft;       /* FFT length N: a power of two, 16..2^24; samples n_samples..N-1 are zero */
    double fs;           /* sampling rate [Hz] */
    double f_low;        /* lower cutoff f_* [Hz] (> 0): the template is zero for f <= f_low (Sec. II.B) */
    double f_high;       /* upper cutoff [Hz]: the template is zero for f > f_high (Sec. II.B) */
    int32_t max_batch;   /* particles per internal chunk (0 = automatic); bounds scratch memory */
    int32_t flags;       /* 0 or FCAS_SETUP_LAZY_SCRATCH */
} fcas_setup;

/* fcas_setup.flags: do not allocate the fitness scratch at create (a context that only takes part
 * in a group uses the group's shared scratch; fcas_fitness allocates it on first use). */
#define FCAS_SETUP_LAZY_SCRATCH 1

typedef struct fcas_ctx fcas_ctx;

/*
 * fcas_create -- prepare a data segment (Sec. II.D).
 *   setup : segment description (host).
 *   det   : [n_det] detector geometry (host).
 *   psd   : [n_det][n_fft/2+1] one-sided PSD S_n^i(f_k), f_k = k fs / n_fft (host or device), or
 *           NULL for the analytic fit to the aLIGO design sensitivity for every detector (Sec. II.A
 *           noise model), S(f) = 1e-49 [x^-4.14 - 5 x^-2 + 111 (1 - x^2 + x^4/2) / (1 + x^2/2)],
 *           x = f / 215 Hz, evaluated in binary64 on the device.
 *           Only bins with f_low < f_k <= f_high, 0 < k < n_fft/2 are read; they must be finite and > 0.
 *   data  : [n_det][n_samples] real strain time series x^i (host or device).
 * The segment is zero-padded to n_fft, transformed (x~[k] = dt sum_n x[n] e^{-2 pi i k n/N}),
 * over-whitened (x~/S, Sec. II.D) and stored on the device together with the template norms
 * <h_c|h_c>^i (Sec. II.D). The call is synchronous. On success *out receives a new context.
 */
int fcas_create(fcas_ctx** out, const fcas_setup* setup, const fcas_detector* det,
                const double* psd, const double* data, void* stream);

/*
 * fcas_create_time_shifted -- fcas_create on a time-shifted copy of the data: detector i's series is
 * first shifted circularly within its n_samples samples, x'_i[t] = x_i[(t - shifts[i]) mod n_samples]
 * (shifts taken modulo n_samples, negative values allowed). Sec. V generates background noise
 * realisations this way: unphysical relative shifts (>= 10 s there) between the detectors' series
 * of one data realisation. The caller's data is not modified. shifts: host array [n_det]; other
 * arguments, errors and synchronisation as fcas_create (FCAS_ERR_INVALID for NULL shifts).
 */
int fcas_create_time_shifted(fcas_ctx** out, const fcas_setup* setup, const fcas_detector* det, const double* psd,
                             const double* data, const int64_t* shifts, void* stream);

/*
 * fcas_fitness -- coherent fitness of a batch of particles (Sec. II.C, eq. gammaSqd).
 *   n       : number of particles (0 is a no-op).
 *   theta   : [n][4] = (alpha [rad, ECEF azimuth], delta [rad, latitude in -pi/2..pi/2],
 *             tau0 [s], tau1.5 [s]) (host or device). tau0 and tau1.5 must be > 0.
 *   fitness : [n] Gamma^2 = max over t in [0, n_samples) of Gamma^2(t) (host or device).
 *   tc      : [n] argmax sample index t (lowest index on ties); the coalescence time at the ECEF
 *             origin is t / fs (host or device).
 * A particle given on the device with a non-finite or non-positive chirp time gets fitness NaN
 * and tc -1; given on the host the whole call fails with FCAS_ERR_INVALID instead.
 */
int fcas_fitness(fcas_ctx* ctx, int64_t n, const double* theta, double* fitness, int64_t* tc,
                 void* stream);

/*
 * fcas_fitness_noalloc -- the same evaluation as fcas_fitness, for callers that cannot allocate
 * device memory while they run. (The paper has no counterpart: this entry point exists for how the
 * library is deployed, not for the method.)
 *
 * Who needs it: programs whose device memory is handed out by another runtime's pool and that may
 * not call cudaMalloc themselves, and analysis loops that fix their memory footprint at start-up
 * because an allocation that fails or stalls in mid-run would lose data. Such a caller creates the
 * context during its set-up phase (fcas_create allocates) and evaluates particles with this call.
 * fcas_fitness may allocate on a call (its particle buffers grow with the batch, host arrays
 * are staged); this call allocates nothing: it calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *
 * Its scratch (per-particle parameters, the intermediate transform between the two FFT passes and
 * the argmax partials) lives in one static device array of 32 MiB inside libfcas.so. The array
 * belongs to the library's no-alloc module, which CUDA loads on a device lazily: the first call of
 * this entry point on a device loads it there, and that load allocates the 32 MiB, which the device
 * then holds until the process exits. Make that first call during the caller's set-up phase, with
 * the context's device current and before any stream capture; from then on the call allocates
 * nothing. One particle needs 2 * n_fft * (8 bytes FP32, 16 bytes FP64 and float-float) plus
 * ~0.6 KB; particles are processed in chunks that fit. A context whose single particle does not fit
 * (n_fft >= 2^21 in FP32, >= 2^20 in the other forms) is rejected with FCAS_ERR_INVALID and a
 * message naming the sizes.
 *
 *   ctx, n, theta, fitness, tc : as for fcas_fitness, except that theta [n][4], fitness [n] and
 *                                tc [n] must be device memory of the current device (host arrays
 *                                would need staging memory): FCAS_ERR_INVALID otherwise. The
 *                                library cannot see the arrays' sizes: the caller guarantees them.
 *   stream                     : a stream of the current device, as for fcas_fitness; the call is
 *                                asynchronous on it.
 * The context's device must be current (FCAS_ERR_INVALID otherwise, as for every entry point that
 * takes a context). The first call on a device also looks up the device address of the scratch
 * array (once per device, with that device current). Every call, from every context and thread,
 * shares the one array and leaves its contents behind; nothing in it needs to start at zero because
 * each call writes every word it reads. Calls that overlap on the GPU (different streams, or
 * different host threads) race on the array: serialise them.
 */
int fcas_fitness_noalloc(const fcas_ctx* ctx, int64_t n, const double* theta, double* fitness, int64_t* tc,
                         void* stream);

/*
 * Particle swarm optimisation (Sec. III): lbest PSO on a ring of particle indices, a fixed number of
 * iterations, best-of-M independent runs with independent random streams. Details the paper defers
 * to earlier work, as implemented here:
 *  - positions normalised to [0,1]^4 and mapped linearly onto the box (alpha, delta, tau0, tau1.5);
 *  - inertia w falls linearly from w_start to w_end over the iterations; every velocity component
 *    is clamped to [-vmax, vmax];
 *  - the neighbourhood of particle p is p and n_neighbours particles on each side (ring); its local
 *    best is the best personal best there (lowest index on ties);
 *  - a particle outside the box is not evaluated (its fitness counts as -inf: "let them fly");
 *  - x0 ~ U[0,1]^4, v0 = clamp(u' - x0) with u' ~ U[0,1]^4;
 *  - one iteration = evaluate, update personal bests, update local bests, move:
 *      v <- clamp(((w v + (c1 r1)(pbest - x)) + (c2 r2)(lbest - x))),  x <- x + v
 *    in binary64, in this order, without fused multiply-adds (bitwise reproducible);
 *  - random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed, counter
 *    (run, iteration, particle, stream) with stream 0 -> r1 / x0, 1 -> r2 / u'; the initial draws
 *    use iteration 0xFFFFFFFF; uniforms are (u + 1/2) 2^-32.
 */
typedef struct fcas_pso_config {
    int32_t n_runs;         /* independent runs, >= 1 */
    int32_t n_particles;    /* particles per run, 1..1024 (the paper uses 40) */
    int32_t n_iter;         /* iterations per run, >= 1 */
    int32_t n_neighbours;   /* ring neighbours on each side, >= 0 (1: two neighbours, as in the paper) */
    uint64_t seed;          /* Philox key */
    double box[8];          /* alpha lo, hi, delta lo, hi [rad], tau0 lo, hi, tau1.5 lo, hi [s] */
    double w_start, w_end;  /* inertia schedule */
    double c1, c2;          /* cognitive and social weights */
    double vmax;            /* velocity clamp (normalised units) */
} fcas_pso_config;

/* Device arrays of the swarm state, rows ordered run-major ([run * n_particles + p]). */
typedef struct fcas_pso_state {
    double* x;              /* [rows][4] normalised positions */
    double* v;              /* [rows][4] velocities */
    double* pbest_x;        /* [rows][4] personal-best positions */
    double* pbest_f;        /* [rows] personal-best fitness (-inf before the first evaluation) */
    int64_t* pbest_tc;      /* [rows] t_c sample index at the personal best (-1 if none) */
} fcas_pso_state;

typedef struct fcas_search_result {
    double fitness;         /* best Gamma^2 of the run (its largest personal best) */
    double theta[4];        /* where: (alpha, delta, tau0, tau1.5) */
    int64_t tc;             /* its argmax t_c sample index */
    int64_t evaluations;    /* fitness evaluations the run performed (particles inside the box) */
} fcas_search_result;

/* Initial positions, velocities and empty personal bests of every run (device state). Asynchronous. */
int fcas_pso_init(const fcas_pso_config* cfg, const fcas_pso_state* state, void* stream);

/*
 * One PSO iteration `iter` (0-based) given the fitness and tc of the current positions
 * (device arrays [rows]; entries of particles outside the box are ignored): personal bests, local
 * bests, then the move. Asynchronous.
 */
int fcas_pso_update(const fcas_pso_config* cfg, int32_t iter, const double* fitness, const int64_t* tc,
                    const fcas_pso_state* state, void* stream);

/*
 * Parameters (alpha, delta, tau0, tau1.5) of normalised positions x [rows][4] (device), written to
 * theta [rows][4] (device); NaN for a particle outside the box (fcas_fitness then skips it).
 * Asynchronous.
 */
int fcas_pso_theta(const fcas_pso_config* cfg, const double* x, double* theta, void* stream);

/*
 * fcas_condition_number -- condition number of the antenna-pattern matrix F(alpha, delta, psi) of the
 * context's network at each particle's sky position (Sec. V relates the ill-posedness of the network
 * problem, and the splitting of the sky-error region, to it): the ratio of the largest to the
 * smallest singular value of the D x 2 matrix, independent of psi.
 *   theta : [n][4] particles (only alpha, delta are read) (host or device).
 *   kappa : [n] condition numbers (host or device); +inf when F is numerically of rank one
 *           (det(F^T F) < 1e-12 (tr(F^T F)/2)^2, the rule the projection uses for G: one detector, or
 *           all detectors seeing the same polarisation), NaN for a non-finite angle.
 * Asynchronous when both arrays are on the device, synchronous otherwise.
 */
int fcas_condition_number(fcas_ctx* ctx, int64_t n, const double* theta, double* kappa, void* stream);

/*
 * fcas_search -- the full search on the context's data: n_runs x n_particles particles evolve
 * together on the device for n_iter iterations; every iteration (positions -> parameters,
 * fitness, update) is one CUDA-graph launch with no host round trip. results: host array
 * [n_runs]. Synchronous.
 */
int fcas_search(fcas_ctx* ctx, const fcas_pso_config* cfg, fcas_search_result* results, void* stream);

/*
 * fcas_gradient -- d Gamma^2 / d theta at a fixed t_c (the argmax returned by fcas_fitness:
 * envelope theorem, the maximisation over t_c is held fixed), theta = (alpha, delta, tau0, tau1.5).
 *   theta : [n][4] (host or device);  tc : [n] t_c sample index (host or device);
 *   grad  : [n][4] (d/d alpha, d/d delta, d/d tau0, d/d tau1.5) of Gamma^2 [per rad, per s]
 *           (host or device).
 * The six band sums each detector needs at t_c (Z, sum k Q, and the four chirp-basis moments)
 * are reduced in binary64; the per-particle combination (antenna patterns, delays, G^-1 and
 * the chirp coefficients, differentiated analytically) is binary64. Particles with invalid input,
 * tc < 0, or an ill-conditioned G (the rank-1 rule of fcas_fitness) get NaN.
 */
int fcas_gradient(fcas_ctx* ctx, int64_t n, const double* theta, const int64_t* tc, double* grad, void* stream);

/*
 * fcas_polish -- gradient polishing of a batch of points (the differentiation form: a few ascent
 * steps along the adjoint gradient of fcas_gradient, e.g. on the best particle of each PSO run of
 * Sec. III; the paper's own search has no such step). Per particle and step, with
 * s = scales * (1, 1, tau0, tau1.5) (absolute step scales for the angles, relative ones for the chirp
 * times), the direction is d = s^2 g / |s g| for the gradient g at the current point and its argmax
 * t_c; trial points theta + l d with l = 1, 1/2, 1/4, ... (at most max_halvings trials) are evaluated
 * with the context's fitness, and the first trial that raises the fitness is taken. A particle whose
 * gradient is not finite, or whose trials all fail, keeps its point for that step.
 *   theta    : [n][4] in: starting points, out: polished points (host or device).
 *   fitness  : [n] out: fitness at the polished points (host or device).
 *   tc       : [n] out: their argmax sample index (host or device).
 *   steps    : ascent steps (>= 0; 0 only evaluates the fitness).
 *   scales   : host [4] step scales (finite, > 0), or NULL for (1e-2 rad, 1e-2 rad, 1e-4, 1e-4).
 *   max_halvings : trial points per step (>= 1).
 *   accepted : [n] out: accepted steps per particle (host or device), or NULL.
 * Synchronous. Every evaluation, gradient, trial and acceptance runs on the device; the host only
 * reads, after each round of trials, how many particles are still searching.
 */
int fcas_polish(fcas_ctx* ctx, int64_t n, double* theta, double* fitness, int64_t* tc, int32_t steps,
                const double* scales, int32_t max_halvings, int32_t* accepted, void* stream);

/*
 * fcas_autotune -- choose the launch shapes of the fitness path for this context by timing them:
 * the N = n1 n2 split (balanced, or a pass-A transform half as long), the number of columns per
 * pass-A CTA among the compiled widths, pass A's stage radix (16, or 8 with twice the threads),
 * and how many adjacent column blocks of a particle are scheduled together (1, 4, 8, 16). Each candidate evaluates n_particles particles (one warm-up,
 * three timed launches, CUDA events); the fastest is kept (the spectrum is laid out again for it).
 * cache_path (may be NULL): a text file of earlier results keyed by GPU name, n_fft, n_det,
 * precision and n_particles; a hit is applied without timing, a miss is timed and appended.
 * Synchronous.
 */
int fcas_autotune(fcas_ctx* ctx, int64_t n_particles, const char* cache_path, void* stream);

/*
 * Groups: several prepared segments (e.g. noise realisations of different durations, so different
 * n_fft) searched together. The contexts share one scratch pool sized for the largest; every PSO
 * iteration of every segment's swarm is one CUDA-graph launch that runs all segments' parameter,
 * fitness and update kernels back to back. The contexts stay owned by the caller and must outlive
 * the group; create them with FCAS_SETUP_LAZY_SCRATCH to avoid per-context scratch.
 */
typedef struct fcas_group fcas_group;

/*
 * fcas_set_shape -- pin the launch shape without timing: split_bias 0 or 1, k1b one of the compiled
 * pass-A widths for the resulting length (0 = default), sub a power of two, radix_bits_a 4 (radix-16
 * stages), 3 (radix-8 stages: the FP32 form's 2^10..2^11-point columns with k1b = 4 and
 * 2^10..2^12-point columns with k1b = 2; the float-float form's 2^10..2^12-point columns with
 * k1b = 2; not the binary64 form) or 0 (the default of the form and length: radix 8 for the
 * float-float form's 2^11-point columns, radix 16 otherwise).
 * FCAS_ERR_INVALID for a shape that is not available. Synchronous.
 */
int fcas_set_shape(fcas_ctx* ctx, int32_t split_bias, int32_t k1b, int32_t sub, int32_t radix_bits_a, void* stream);

/* max_batch: particles per chunk of the shared scratch (0 = automatic, <= 64). */
int fcas_group_create(fcas_group** out, int32_t n_ctx, fcas_ctx* const* ctxs, int32_t max_batch);

/*
 * fcas_group_search -- one swarm of cfg per segment (segment s draws its random numbers with the
 * key seed + s * 0x9E3779B97F4A7C15), all advanced together for cfg->n_iter iterations.
 * results: host array [n_ctx][n_runs]. Synchronous.
 */
int fcas_group_search(fcas_group* group, const fcas_pso_config* cfg, fcas_search_result* results, void* stream);

/*
 * fcas_group_search_boxes -- fcas_group_search with one PSO box per segment: segment s searches
 * boxes[8 s .. 8 s + 7] (the layout of fcas_pso_config.box) instead of cfg->box, with the same
 * per-segment random-number key. A context may appear in a group several times, so one data
 * segment can be searched over several rectangles of the (tau0, tau1.5) plane together (Sec. IV:
 * the rectangles covering the chirp-time range are searched in parallel, their number does not
 * add to the run time). boxes: host array [n_ctx][8]; each box is validated like cfg->box
 * (FCAS_ERR_INVALID names the segment). results: host array [n_ctx][n_runs]. Synchronous.
 */
int fcas_group_search_boxes(fcas_group* group, const fcas_pso_config* cfg, const double* boxes,
                            fcas_search_result* results, void* stream);

void fcas_group_destroy(fcas_group* group);

/*
 * fcas_tau_tiles -- n0 x n15 overlapping rectangles covering [tau0_lo, tau0_hi] x [tau15_lo, tau15_hi]
 * (Sec. IV covers the chirp-time range with overlapping rectangles searched in parallel). Along each
 * axis the n tiles have width w = (hi - lo) / (n - (n - 1) overlap) and tile j starts at
 * lo + j (1 - overlap) w, so neighbours share the fraction `overlap` of a width and the last tile
 * ends at hi. Written as PSO boxes over the whole sky (alpha in [0, 2 pi], delta in [-pi/2, pi/2])
 * to boxes[8 (j0 n15 + j15) ...], j0 the tau0 index. Needs 0 < lo < hi on both axes, n0, n15 >= 1,
 * 0 <= overlap < 1 (FCAS_ERR_INVALID otherwise). boxes: host array [n0 n15][8]. Host only.
 */
int fcas_tau_tiles(double tau0_lo, double tau0_hi, double tau15_lo, double tau15_hi, int32_t n0, int32_t n15,
                   double overlap, double* boxes);

/* Release every resource held by the context (NULL is a no-op). Synchronises the device. */
void fcas_destroy(fcas_ctx* ctx);

/* Message of the last failure on the calling thread ("" if none). Valid until the next call. */
const char* fcas_last_error(void);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int fcas_version(void);

/* Layout and size facts of a context, for benchmarks and tests. */
typedef struct fcas_info {
    int64_t n_fft, n1, n2;      /* N = n1 * n2: pass A transforms length n2, pass B length n1 */
    int64_t k_lo, k_hi;         /* first and last template bin */
    int64_t n_band;             /* k_hi - k_lo + 1 */
    int64_t chunk;              /* particles per internal chunk */
    int32_t n_det, precision;
    double scale;               /* power of two applied to the whitened data (Gamma^2 is invariant) */
    double sigma2[FCAS_MAX_DET];/* unscaled template norms <h_c|h_c>^i */
    int64_t inter_bytes;        /* bytes per particle that cross HBM between the two FFT passes */
    int64_t series;             /* length-N transforms per particle (2: the network-weighted series) */
    int32_t split_bias;         /* n2 = 2^(floor(log2 n_fft / 2) - split_bias) */
    int32_t k1b;                /* pass-A columns per CTA */
    int32_t sub;                /* pass-A column blocks of a particle scheduled together */
    int32_t radix_bits_a;       /* pass-A full-stage radix: 4 (radix 16) or 3 (radix 8, twice the threads) */
    double tuned_ms_per_particle; /* time per particle of the tuned shape (0: not tuned) */
} fcas_info;

int fcas_get_info(const fcas_ctx* ctx, fcas_info* info);

/*
 * Kernel timing: when enabled, every kernel launched by fcas_fitness is bracketed by CUDA events
 * on the launching stream. fcas_profile_read synchronises those events and returns, for one
 * kernel kind, the summed device time [ms] and the number of launches since the last enable.
 */
enum fcas_kernel_kind {
    FCAS_KERNEL_GEOMETRY = 0,   /* per-particle sky geometry, chirp coefficients, G^-1 */
    FCAS_KERNEL_PASS_A = 1,     /* fused template x data x delay phase + first FFT pass */
    FCAS_KERNEL_PASS_B = 2,     /* second FFT pass + antenna projection + partial argmax */
    FCAS_KERNEL_REDUCE = 3,     /* final argmax across CTAs */
    FCAS_KERNEL_KINDS = 4
};

int fcas_profile_enable(fcas_ctx* ctx, int on);
int fcas_profile_read(fcas_ctx* ctx, int kind, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* FCAS_H */
