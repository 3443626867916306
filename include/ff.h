/*
 * ff.h - C interface of the GB300 ferrofluid library (libff.so).
 *
 * The library evaluates the long-range dipole-dipole field and force on N
 * magnetic particles by a Barnes-Hut octree and advances positions and
 * moments by the Langevin equations, following Polyakov et al.,
 * "Large-scale Ferrofluid Simulations on Graphics Processing Units"
 * (arXiv:1212.2934): model in Sec. 2, all-pairs and Barnes-Hut schemes in
 * Sec. 3, Euler-Maruyama integration in Sec. 4, magnetisation observables in
 * Sec. 5.  All quantities are in the paper's reduced units, with lengths
 * measured in hard-core diameters (the dipolar terms carry the factor
 * dip_scale).
 *
 * Conventions for every call:
 *  - Return value: an ff_status; the library never aborts.  On failure
 *    ff_last_error(ctx) gives a message.  After FF_ECUDA or FF_EDEVICE the
 *    context is poisoned and every call except ff_destroy, ff_last_error and
 *    ff_set_particles returns FF_ESTATE.
 *  - Arrays passed in or out are n x 3, row-major (x, y, z of particle 0,
 *    then particle 1, ...), in the caller's particle order, of element type
 *    `dtype` (FF_DTYPE_F32 = float, FF_DTYPE_F64 = double) and located in
 *    host memory (loc = FF_HOST, any host pointer) or device memory of the
 *    context's GPU (loc = FF_DEVICE).  The library copies what it reads and
 *    writes only what it is asked to; the caller keeps ownership.
 *  - Device work runs on the context's stream in order.  ff_step returns
 *    before the GPU finishes; every call that hands results to the caller
 *    waits for them.
 *  - One context must not be used from two host threads at once.
 */
#ifndef FF_H
#define FF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ff_ctx ff_ctx; /* opaque; owns all of its device memory */

typedef enum {
    FF_OK = 0,
    FF_EINVAL = 1,     /* bad argument (pointer, size, enum, parameter range) */
    FF_ENOMEM = 2,     /* device or host allocation failed */
    FF_ECUDA = 3,      /* a CUDA runtime call failed */
    FF_EDEVICE = 4,    /* a kernel raised its error flag (iteration guard) */
    FF_ENONFINITE = 5, /* a position was NaN or infinite */
    FF_ESTATE = 6      /* call not valid now: no particles set, or poisoned */
} ff_status;

/*
 * FF_FP32: state, tree, traversal and integration in IEEE single (the
 * paper's choice, Sec. 4).  FF_FP64: everything in double.  FF_MIXED: as
 * FF_FP32, except that the cell aggregation (Eq. magCenter) sums positions
 * and moments in double and rounds each centre (double sum / count) and each
 * moment sum to single once.  Energies and magnetisation are summed in double
 * in every mode.
 */
typedef enum { FF_FP32 = 0, FF_FP64 = 1, FF_MIXED = 2 } ff_precision;
typedef enum { FF_ALGO_BH = 0, FF_ALGO_AP = 1 } ff_algo;
typedef enum { FF_DTYPE_F32 = 0, FF_DTYPE_F64 = 1 } ff_dtype;
typedef enum { FF_HOST = 0, FF_DEVICE = 1 } ff_loc;

/*
 * Run parameters (reduced units of Sec. 2).  Fill with ff_params_default
 * and change what differs.  struct_size must be sizeof(ff_params).
 */
typedef struct {
    uint32_t struct_size;
    int32_t precision;     /* ff_precision of state, tree and arithmetic */
    int64_t n;             /* particle count, 1 .. 2^27 */
    int32_t algo;          /* ff_algo used by ff_step and ff_energy */
    int32_t leaf_max;      /* most particles in a leaf cell, 1..64 (paper: 1, Sec. 3.2) */
    double theta;          /* opening angle >= 0; 0 sums every pair exactly */
    double dt;             /* Euler-Maruyama step (paper: 1e-3, Sec. 4) */
    double gamma_t;        /* translational friction Gamma_t (Sec. 2) */
    double gamma_r;        /* rotational friction Gamma_r (Sec. 2) */
    double inertia;        /* reduced moment of inertia (2/5, Sec. 2) */
    double kT;             /* reduced thermal energy */
    double rot_noise;      /* rotational noise factor c_r: <xi xi> = c_r kT Gamma_r (2) */
    double dip_scale;      /* prefactor of the dipolar field and force */
    double lj_eps;         /* LJ epsilon (Sec. 2, Eq. LJ); 0 turns LJ off */
    double lj_sigma;       /* LJ sigma: the force vanishes at this distance */
    double lj_rcut;        /* LJ cut-off radius (> 0 when lj_eps != 0) */
    double h_ext[3];       /* applied field */
    double box_lo[3];      /* container: wall planes at box_lo - 1/2 ... */
    double box_hi[3];      /* ... and box_hi + 1/2 */
    int32_t walls;         /* 1: LJ-type walls on the container faces */
    int32_t device;        /* CUDA device ordinal */
    double wall_eps;       /* wall epsilon */
    uint64_t seed;         /* Philox key of the thermal noise */
    int32_t count_interactions; /* 1: record per-particle interaction counts */
    int32_t traverse_group;  /* lanes walking the cell list together: 1,2,4,8,16,32; 0 = default.
                                Results do not depend on it (every lane decides for itself). */
    void *stream;          /* cudaStream_t to run on; NULL: the context creates one */
    int32_t rotation;      /* FF_ROT_VECTOR (default): rigid rotor I w' = u x h - G_r w + noise,
                              u' = w x u; FF_ROT_PRINTED: the printed reduced angle equations
                              (theta, phi and their rates; the rates kept in w_x, w_y), which
                              do not relax toward the Boltzmann distribution (Sec. 2) */
    int32_t quadrupole;    /* 1: every accepted cell also contributes its dipole-position
                              (quadrupole) term about the centre, -grad Phi to h and -H Phi u
                              to f with Phi = (3 r.S.r - m r^2)/r^5, S and m from
                              sum (rho_i - c) (x) u_i: an accuracy option beyond the paper's
                              pseudo-particles (error second order in theta).  Barnes-Hut
                              only; not with ff_energy_grad or ff_mz_sensitivity */
} ff_params;

enum { FF_ROT_VECTOR = 0, FF_ROT_PRINTED = 1 };

/* Energies and observables returned by ff_energy (FP64). */
typedef struct {
    double e_dip;      /* -1/2 sum_k u_k . h_dip_k */
    double e_zeeman;   /* -sum_k u_k . h_ext */
    double e_sr;       /* LJ pair energy (each pair once), shifted to 0 at rcut */
    double e_wall;     /* wall energy */
    double e_kin_t;    /* 1/2 sum v^2 */
    double e_kin_r;    /* I/2 sum w^2 */
    double m[3];       /* <u> = (1/N) sum u (Sec. 5) */
    double hdip_z_mean;/* (1/N) sum h_dip_z (Sec. 5) */
} ff_energy_t;

/* Size of the last tree and interaction totals (ff_tree_info). */
typedef struct {
    int64_t ncells;        /* cells of the last tree */
    int32_t depth;         /* deepest cell level (root = 0) */
    int32_t reserved;
    double root[4];        /* root cube: lower corner x, y, z and side */
    int64_t interactions;  /* sum over particles of accepted cells + exact pairs (counting on) */
    int64_t accepted;      /* sum of accepted cells */
    int64_t pairs;         /* sum of exact pairs */
    int64_t opened;        /* sum of opened cells */
} ff_tree_info_t;

/* Fills *p with defaults: FP32, BH, theta 0.5, leaf_max 1, dt 1e-3,
 * gamma_t = gamma_r = 0.1, inertia 0.4, kT 1, rot_noise 2, dip_scale 1,
 * LJ eps 1 sigma 1 rcut 2.5, no field, no walls, device 0, seed 1. */
void ff_params_default(ff_params *p);

/*
 * Creates a context for p->n particles on p->device (Sec. 2 model, Sec. 3
 * schemes) and allocates its device memory: about 0.5 KB per particle in FP32
 * and 0.8 KB in FP64 (66 GB and 110 GB at n = 2^27), gradient buffers apart.
 * The tree's cell arrays start with room for 2 n + 8192 cells (gases, chains
 * and dense packings use 1.2 to 1.8 cells per particle).  A build that needs
 * more raises a device flag instead of writing past them; that step and the
 * ones after it leave the state unchanged, and the next call that waits for
 * results grows the arrays (to 1.25 x the need, at most 22 n + 1, the most any
 * tree can have), runs the held-back steps again and completes: results are
 * those of a context that had the room from the start.  *out receives the
 * context.  FF_EINVAL for out-of-range parameters, FF_ENOMEM, FF_ECUDA;
 * the reason is then given by ff_last_error(NULL).
 */
ff_status ff_create(const ff_params *p, ff_ctx **out);

/* Frees the context and its memory; NULL is allowed. */
ff_status ff_destroy(ff_ctx *ctx);

/*
 * Sets the state of Sec. 2 (positions rho_k, unit moments u_k, velocities,
 * angular velocities) from n x 3 arrays; vel and omega may be NULL (zero).
 * Moments are used as given (the caller normalises them).  Clears a
 * poisoned state.  Waits until the copy is done.
 */
ff_status ff_set_particles(ff_ctx *ctx, const void *pos, const void *u, const void *vel,
                           const void *omega, int32_t dtype, int32_t loc);

/* Copies the current state into n x 3 arrays (any pointer may be NULL). Waits. */
ff_status ff_get_particles(ff_ctx *ctx, void *pos, void *u, void *vel, void *omega,
                           int32_t dtype, int32_t loc);

/*
 * Field and force of the current state (Sec. 3): h_out = dip_scale * sum of
 * the reduced dipolar fields h_kj (Sec. 2, Eq. h_dip, h_ext excluded) and
 * f_out = dip_scale * dipolar force (Eq. f_dip) plus, if include_sr, the LJ
 * force (Eq. LJ) of pairs closer than lj_rcut.  algo = FF_ALGO_AP sums every
 * pair (Sec. 3.1, Algorithm 1); FF_ALGO_BH uses the octree (Sec. 3.2) with
 * opening angle theta: a cell stands in for its particles (moment sum at
 * their geometric centre, Eq. magCenter) iff the particle is not in it,
 * side^2 < theta^2 |rho_k - centre|^2, and (LJ on) the cell's cube is at
 * least lj_rcut away.  Either output pointer may be NULL.  Waits.
 */
ff_status ff_dipolar_field(ff_ctx *ctx, int32_t algo, double theta, int32_t include_sr,
                           void *h_out, void *f_out, int32_t dtype, int32_t loc);

/*
 * Advances nsteps >= 0 Euler-Maruyama steps of dt (Sec. 4) of the Langevin
 * equations (Sec. 2; rotation in vector form) with the context's algorithm
 * and theta: per step tree build, field, walls, Philox noise keyed by
 * (seed, step, particle) and the update of positions, velocities, moments
 * and angular velocities.  Returns without waiting; errors raised on the GPU
 * are reported by the next waiting call.
 */
ff_status ff_step(ff_ctx *ctx, int64_t nsteps);

/*
 * Energies and the Sec. 5 observables of the current state, in FP64, with
 * the field of the context's algorithm.  Waits.
 */
ff_status ff_energy(ff_ctx *ctx, ff_energy_t *out);

/* Step counter (the noise of step s is drawn with counter s). */
ff_status ff_get_step(const ff_ctx *ctx, int64_t *step);
ff_status ff_set_step(ff_ctx *ctx, int64_t step);

/*
 * Batched ensembles: splits the n particles into nsys independent systems
 * (particles 0 .. counts[0]-1 form system 0, the next counts[1] system 1,
 * and so on, in the caller's order), each with its own root cube and tree
 * (Sec. 3.2), its own applied field h_ext[3*s .. 3*s+2] and, when walls are
 * on, its own container box_lo/box_hi[3*s ..] (NULL: the context's field or
 * box for every system).  Systems never interact; every other parameter is
 * shared.  This is how the magnetisation curves of Sec. 5 are run: many
 * ensembles at different field amplitudes advanced together, one CUDA graph
 * per step for all of them.  nsys = 1 .. 65536, counts >= 1 summing to n.
 * All-pairs evaluation is not available for batched systems.  Waits.
 */
ff_status ff_set_systems(ff_ctx *ctx, int32_t nsys, const int64_t *counts, const double *h_ext,
                         const double *box_lo, const double *box_hi);

/*
 * Per-system sums accumulated by ff_step since the last reset (or since
 * ff_set_systems): out[4*s + q] = sum over steps and over the particles of
 * system s of u_x, u_y, u_z (q = 0..2) and h_dip_z (q = 3), taken from the
 * state at the start of each step (Sec. 5: <u> and <h_dip_z> follow by
 * dividing by steps x particles).  *nsteps receives the number of steps.
 * reset = 1 clears the sums afterwards.  The sums are formed with FP64
 * atomics, so their last bits may differ between runs.  Waits.
 */
ff_status ff_system_moments(ff_ctx *ctx, double *out, int64_t *nsteps, int32_t reset);

/*
 * Traversal schedule autotuner.  The per-particle walk (Sec. 3.2, kernel 5)
 * can be run with G = 1, 2, 4, 8, 16 or 32 lanes walking the cell list
 * together; every G gives bit-identical fields and forces (each lane makes its
 * own particle's decisions in depth-first order), only the speed differs with
 * the workload.  This sorts the current state and builds the tree once (like
 * ff_dipolar_field with the context's theta, LJ included), then times `reps`
 * traversals for each candidate with CUDA events on the context's stream and
 * keeps the fastest (minimum over reps; ties to the earlier candidate) as the
 * context's traverse_group for later ff_step and ff_dipolar_field calls.
 * groups[ngroups]: candidates (each one of 1, 2, 4, 8, 16, 32), or NULL with
 * ngroups = 0 for all six.  reps = 1 .. 100.  *best_group receives the choice;
 * ms (may be NULL) receives ngroups (6 for NULL groups) per-candidate times in
 * milliseconds.  Barnes-Hut contexts only.  Waits.
 */
ff_status ff_tune_traversal(ff_ctx *ctx, const int32_t *groups, int32_t ngroups, int32_t reps,
                            int32_t *best_group, float *ms);

/*
 * Launch schedules of the traversal (no counterpart in the paper; Sec. 3.2
 * kernel 5 ran one fixed launch on its GPU).  Schedule i = 1 ..
 * ff_schedule_count() is a lane group (as traverse_group) with, for the plain
 * single-precision walk (interaction counting off, no dipole-position terms),
 * its own compiled block shape: threads per block and the resident blocks per
 * SM the kernel's register budget is set for; other walks use their group's
 * default shape.  The traversal is persistent (as many blocks as fit), so the
 * shape trades registers per thread against resident warps.  Every schedule
 * gives bit-identical fields and forces (each lane decides and sums for its own
 * particle in depth-first order).  ff_schedule_info fills the three numbers
 * (any pointer may be NULL); FF_EINVAL for an index out of range.
 */
int32_t ff_schedule_count(void);
ff_status ff_schedule_info(int32_t index, int32_t *group, int32_t *threads,
                           int32_t *blocks_per_sm);

/*
 * Makes schedule `index` (0: traverse_group with its default shape) the
 * context's traversal launch for later ff_step and ff_dipolar_field calls.
 * FF_EINVAL for an index out of range.
 */
ff_status ff_set_schedule(ff_ctx *ctx, int32_t index);

/*
 * Schedule autotuner: sorts the current state and builds the tree once (as
 * ff_dipolar_field with the context's theta, LJ included), times `reps`
 * traversals (1 .. 100) with every schedule by CUDA events on the context's
 * stream, and keeps the fastest (minimum over reps; ties to the lower index)
 * as the context's schedule.  *best_schedule receives it; ms (may be NULL)
 * receives ff_schedule_count() times in milliseconds, schedule 1 first.
 * Barnes-Hut contexts only.  Waits.
 */
ff_status ff_tune_schedule(ff_ctx *ctx, int32_t reps, int32_t *best_schedule, float *ms);

/*
 * Dipolar energy E = -1/2 sum_k u_k . h_k (Sec. 5; h from algo, LJ excluded)
 * and its gradient with respect to every position and moment.  With
 * FF_ALGO_AP every pair is exact: dE/du = -h and dE/drho = -f (the dipolar
 * force).  With FF_ALGO_BH the gradient is exact for the Barnes-Hut energy
 * with this evaluation's opening decisions frozen (the decisions are
 * piecewise constant in the positions, Sec. 3.2): besides -1/2 h_k and
 * -1/2 f_k it carries the reverse sums over every interaction whose source
 * (an accepted cell, or a particle summed exactly) contains particle k.
 * The current state is evaluated (and, for Barnes-Hut, sorted into key
 * order); *energy (may be NULL) receives E in FP64; grad_pos and grad_u (may
 * be NULL) receive n x 3 values in the caller's order, dtype/loc as in
 * ff_get_particles.  With both NULL only the field and E are computed (the
 * cost of one field evaluation).  The Barnes-Hut gradient keeps every
 * particle's list of sources (4 bytes per interaction, in chunks of 128;
 * 700 to 900 interactions per particle at theta = 0.5) and 8 bytes per
 * interaction of record space, allocated on first use and grown as needed
 * (about 10 KB per particle in all at theta = 0.5); 2^32 - 16 interactions
 * or more (about 5 million particles at theta = 0.5) is FF_EINVAL.  Waits.
 */
ff_status ff_energy_grad(ff_ctx *ctx, int32_t algo, double theta, double *energy, void *grad_pos,
                         void *grad_u, int32_t dtype, int32_t loc);

/*
 * Sensitivity of the mean magnetisation to the applied field (Sec. 5):
 * advances the state by nsteps steps (as ff_step) and returns
 *   Mz = 1/nsteps sum over the nsteps new states of 1/n sum_k u_z,k
 * in *mz and dMz/dh_ext (3 components) in dmz_dh, by reverse mode through
 * every step: the Euler-Maruyama update (Sec. 4, torque, friction and the
 * renormalisation of u; walls), the Barnes-Hut field and force (Sec. 3.2)
 * with each step's opening decisions frozen, and the LJ forces.  The state
 * is saved every `every` steps and each stretch is recomputed on the way
 * back (memory: about nsteps / every + every state copies).  Noise is
 * additive and keyed by (seed, step, particle), so it does not depend on
 * h_ext and the recomputation reproduces it.  Single-system Barnes-Hut
 * contexts; the context ends at the advanced state.  Waits.
 */
ff_status ff_mz_sensitivity(ff_ctx *ctx, int64_t nsteps, int64_t every, double *mz,
                            double *dmz_dh);

/* Waits for the context's stream and reports any error flag raised on the GPU. */
ff_status ff_synchronize(ff_ctx *ctx);

/* Tree size and interaction totals of the last Barnes-Hut evaluation (waits). */
ff_status ff_tree_info(ff_ctx *ctx, ff_tree_info_t *out);

/*
 * Copies the last Barnes-Hut tree to host arrays (any pointer may be NULL):
 * keys[n] (sorted 63-bit Morton keys), order[n] (input index of each sorted
 * position) and, for ncells cells in depth-first preorder, pbegin/pend
 * (sorted particle range), skip (index after the subtree), level, leaf,
 * centre[3*ncells] (geometric centre), moment[3*ncells] (moment sum), in
 * dtype.  Waits.
 */
ff_status ff_get_tree(ff_ctx *ctx, uint64_t *keys, uint32_t *order, int32_t *pbegin,
                      int32_t *pend, int32_t *skip, int32_t *level, int32_t *leaf,
                      void *centre, void *moment, int32_t dtype);

/*
 * Per-particle counts of the last Barnes-Hut evaluation in the caller's
 * order (host arrays of n, any may be NULL): accepted cells, exact pairs and
 * opened cells.  Needs count_interactions = 1.  Waits.
 */
ff_status ff_get_counts(ff_ctx *ctx, int32_t *accepted, int32_t *pairs, int32_t *opened);

/*
 * Stage timing (CUDA events on the context's stream) and launch counting.
 * Stages: 0 keys (root cube + Morton keys), 1 radix sort, 2 gather into key
 * order, 3 tree build, 4 aggregation, 5 field (traversal or all-pairs),
 * 6 integration and observables, 7 output conversion.  ms[i] and calls[i]
 * accumulate the device time and the number of timed executions of stage i;
 * launches counts the kernels this context launched.
 */
typedef struct {
    double ms[8];
    int64_t calls[8];
    int64_t launches;
} ff_profile_t;

/* enable = 1 starts timing and zeroes the counters; 0 stops timing. */
ff_status ff_profile(ff_ctx *ctx, int32_t enable);

/* Waits for the stream and returns the accumulated stage times and launches. */
ff_status ff_profile_read(ff_ctx *ctx, ff_profile_t *out);

/* Message for the last failure on this context (never NULL).  With
 * ctx = NULL: why the last ff_create or ff_morton_order_noalloc on the
 * calling thread failed. */
const char *ff_last_error(const ff_ctx *ctx);

/* Name of a status code. */
const char *ff_status_string(ff_status s);

/*
 * Allocation-free Morton ordering, for callers that cannot allocate device
 * memory: applications whose device memory belongs to their own pool or
 * allocator, and loops that cannot stall on an allocation (cudaMalloc may
 * synchronise the device).  The paper has no counterpart; it is the key-sort
 * stage of the Barnes-Hut path packaged without allocation.  The call reads
 * its error word back to the host and waits for the stream, so it cannot be
 * issued on a stream that is being captured into a graph.
 *
 * pos: device pointer, n x 3 float, caller's order.  Writes keys_out[n]
 * (device, uint64: the sorted 63-bit Morton keys of the root cube of these
 * positions) and order_out[n] (device, uint32: the input index of each sorted
 * position; ties keep input order), exactly as ff_get_tree reports them for a
 * single-precision context.  stream: a cudaStream_t, NULL for the default
 * stream.  Waits for the stream before returning.
 *
 * Nothing is allocated: besides the caller's buffers the work uses one fixed
 * scratch array inside the library, sized for n <= FF_NOALLOC_MAX_N (about
 * 3.7 MB, held on every GPU that loads the library until the process exits).
 * The first call on a device looks up the array's device address and keeps
 * it for the life of the process: make that first call before any stream
 * capture on that device, and do not use the call on a device after
 * cudaDeviceReset.  Every call shares the array: calls whose GPU work
 * overlaps (other streams, other host threads on the same device) race and
 * must not be issued.
 *
 * FF_EINVAL: a NULL pointer, or n outside 1 .. FF_NOALLOC_MAX_N.
 * FF_ENONFINITE: a position is NaN or infinite.  FF_EDEVICE: a sort tile's
 * bounded wait for an earlier tile ran out (the output is then not sorted).
 * FF_ECUDA: a CUDA call failed.  The reason is given by ff_last_error(NULL).
 */
#define FF_NOALLOC_MAX_N 131072
ff_status ff_morton_order_noalloc(const float *pos, int64_t n, uint64_t *keys_out,
                                  uint32_t *order_out, void *stream);

/*
 * Self-test of the key sort's only wait on other thread blocks (no
 * counterpart in the paper).  Each tile of a sort pass adds up the digit
 * counts that earlier tiles publish, polling each word a bounded number of
 * times and raising a device error flag when the polls run out (the host then
 * reports FF_EDEVICE instead of waiting forever).  This call sorts n
 * synthetic keys in buffers it allocates and frees, with the first tile
 * withholding its counts and every word polled once, so the second tile's
 * wait must run out.
 *
 * n: 8192 .. 2^24 (at least two tiles).  stream: a cudaStream_t, NULL for
 * the default stream.  Waits before returning.  FF_OK: the wait ran out and
 * its flag reached the host.  FF_EDEVICE: it did not.  FF_EINVAL: n out of
 * range.  FF_ECUDA: a CUDA call failed.  The reason is given by
 * ff_last_error(NULL).
 */
ff_status ff_selftest_sort_wait(int64_t n, void *stream);

/*
 * Self-test of the other wait on other thread blocks (no counterpart in the
 * paper): the energy gradient's record pass scans the sorted records' entry
 * counts in one pass, each tile adding up the counts that earlier tiles
 * publish, polling a bounded number of times and raising the same device
 * error flag when the polls run out.  This call runs that pass on nrec
 * synthetic records in buffers it allocates and frees, with the first tile
 * withholding its count and every look-back window read once, so the second
 * tile's wait must run out.
 *
 * nrec: 4096 .. 2^24 (at least two tiles).  stream: a cudaStream_t, NULL for
 * the default stream.  Waits before returning.  FF_OK: the wait ran out and
 * its flag reached the host.  FF_EDEVICE: it did not.  FF_EINVAL: nrec out of
 * range.  FF_ECUDA: a CUDA call failed.  The reason is given by
 * ff_last_error(NULL).
 */
ff_status ff_selftest_record_wait(int64_t nrec, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FF_H */
