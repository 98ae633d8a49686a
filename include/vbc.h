/*
 * vbc.h -- C ABI of libvbc.so: the valency-bounding correction (VBC) force and
 * energy evaluation, its cell-list neighbour build and a Langevin integrator,
 * all running as CUDA kernels on one GPU (sm_103a).
 *
 * The method (paper "Valency-bounding correction potential for coarse-grained
 * molecular dynamics simulations", Sec. 2):
 *   omega(x; x1, x2) = 1 (x <= x1), (1 - ((x - x1)/(x2 - x1))^2)^2, 0 (x >= x2)  Eq. (omega)
 *   n_i   = sum_{j != i} omega(r_ij; r_l, r_h)                                 Eq. (counter)
 *   Psi   = omega(n_i; f - delta, f - delta + 1) omega(n_j; f - delta, f - delta + 1)
 *                                                                  Eqs. (Psi), (Psidelta)
 *   V^    = V_r + Psi V_a,  U = sum_{i<j} V^(r_ij)                              Eq. (Vhat)
 *   V_r   = E_r (1 - (r/r_r)^2)^2 for r < r_r;  V_a = -E_a (1 - u^2)^2 for
 *           r_r < r < r_a, u = (r - (r_a + r_r)/2) / ((r_a - r_r)/2)             Eq. (softcore)
 * Forces are -grad U including the chain-rule terms through dPsi/dn (the
 * paper's two passes over the neighbour list, Sec. 2): with s_i the switch of
 * particle i and A_i = s_i' sum_j s_j V_a(r_ij) = dU/dn_i,
 *   F_i = -sum_j [V_r'(r) + s_i s_j V_a'(r) + (A_i + A_j) omega'(r)] (x_i - x_j)/r.
 *
 * Conventions for every call:
 *   - Units are reduced: lengths in r_r (usually 1), energies as given, unit mass.
 *   - Arrays of positions, velocities and forces are row-major [n][3] doubles
 *     in the caller's particle order.  The library keeps its own copy of the
 *     state in device memory it owns (sorted along a Morton curve internally)
 *     and un-permutes every output.  Caller pointers are borrowed for the
 *     duration of the call only.
 *   - `*_on_device` flags say whether caller pointers are device (1) or host
 *     (0) memory.  Host memory may be pageable or pinned.
 *   - All work is enqueued on the system's stream (the one given at creation,
 *     or a stream the library creates).  Calls return after the outputs the
 *     caller asked for are written.
 *   - Return value: VBC_OK (0) or a negative VBC_ERR_* code; no call aborts
 *     the process.  vbc_last_error() gives a message for the calling thread.
 */
#ifndef VBC_H
#define VBC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    VBC_OK = 0,
    VBC_ERR_INVALID_ARG = -1,   /* bad size, parameter, pointer or box */
    VBC_ERR_CUDA = -2,          /* a CUDA runtime call failed (message has the detail) */
    VBC_ERR_OOM = -3,           /* device allocation failed */
    VBC_ERR_NLIST_OVERFLOW = -4,/* neighbour list still overflows after growing to its limit */
    VBC_ERR_UNSTABLE = -5,      /* non-finite position or velocity produced */
    VBC_ERR_TIMEOUT = -6,       /* a wait ended before the awaited work (serving) */
    VBC_ERR_CANCELLED = -7      /* a served request was dropped or stopped by vbc_server_destroy */
};

/* Precision of the pair arithmetic. */
enum {
    VBC_FP32_SPLIT = 0, /* FP32 pair arithmetic on 32-bit fixed-point positions; exact
                           integer squared distances and fixed-point sums for the counts;
                           FP64 state (positions, velocities) and FP64 energy/virial */
    VBC_FP64 = 1        /* FP64 pair arithmetic on 64-bit fixed-point positions */
};

/* VBC(r_l, r_h, delta) on the polynomial soft core (Sec. 2 and Sec. 4 "bond lifetimes").
 * Requirements: 0 < r_r < r_a, 0 <= r_l < r_h, E_r >= 0, E_a >= 0.  The standard VBC
 * is r_r = 1, r_a = r_l = 1.5, r_h = 2, delta = 0; the optimised one is
 * r_l = 1.29, r_h = 1.50, delta = 0.30 (in units of r_r). */
typedef struct {
    double r_r, r_a, r_l, r_h;  /* repulsive range, attractive range, counting radii */
    double E_r, E_a;            /* repulsive barrier height, attractive well depth */
    double f, delta;            /* valency and threshold shift (f may be non-integer) */
} vbc_pair_params;

typedef struct {
    int64_t n;                /* particles, 1 <= n <= 2^31 - 1 */
    double box[3];            /* periodic orthorhombic box edges; VBC_FP32_SPLIT needs a cube.
                                 Each edge must hold >= 3 cells of r_c + skin, where
                                 r_c = max(r_r, r_a, r_h). */
    const double* pos;        /* [n][3] initial positions (any image; unwrapped positions
                                 are tracked from here on) */
    const double* vel;        /* [n][3] initial velocities, or NULL for zeros */
    vbc_pair_params params;
    double skin;              /* Verlet skin; the list radius is r_c + skin (skin > 0) */
    uint64_t seed;            /* key of the Langevin noise (Philox4x32-10) */
    int32_t precision;        /* VBC_FP32_SPLIT or VBC_FP64 */
    int32_t nlist_cap;        /* initial neighbour-list capacity per particle, 0 = automatic */
    void* stream;             /* cudaStream_t to enqueue on, or NULL for a library-owned stream */
    int32_t inputs_on_device; /* pos/vel are device pointers */
} vbc_config;

typedef struct vbc_system vbc_system;

/* Diagnostics of the last evaluation / of the run so far. */
typedef struct {
    int64_t n;
    int64_t step;              /* Langevin steps taken (the noise counter) */
    int64_t rebuilds;          /* neighbour-list builds so far */
    int32_t nlist_cap;         /* current capacity per particle */
    int32_t nlist_max;         /* longest list at the last build */
    double nlist_mean;         /* mean list length at the last build */
    int64_t pairs_within_rc;   /* unordered pairs with r < r_c at the last energy evaluation */
    int64_t in_window;         /* particles with f - delta < n_i < f - delta + 1 (last count pass) */
    int64_t unsaturated;       /* particles the last count pass had to walk in full: fewer than
                                  ceil(f - delta + 1) of their kept near neighbours within r_l */
    int32_t stage_cap;         /* staged particles per cell group (current capacity) */
    int32_t group_cap;         /* particles per cell group (current capacity) */
    int32_t groups;            /* cell groups (units of the list build and of the dense row walks) */
    int64_t capacity_grows;    /* capacity growths after an overflow since creation (each resumes the
                                  interrupted call from the overflowing build) */
    int64_t device_bytes;      /* device memory the system holds at its current capacities */
} vbc_stats;

/*
 * Create a system: copy the configuration in, allocate device memory, build
 * the neighbour list.  On success *out owns everything; release it with
 * vbc_destroy.  Errors: INVALID_ARG (n < 1, non-positive box, box too small,
 * non-cubic box with VBC_FP32_SPLIT, bad parameters, NULL pos/out), OOM, CUDA.
 */
int vbc_create_system(const vbc_config* cfg, vbc_system** out);

/* ---------------------------------------------------------------- several types and bonds
 * Multi-type VBC (Sec. 2: the counter may run over chosen neighbour types
 * only) with harmonic bonds (the bead-spring sticker chains of Sec. 4).  The
 * pair (i, j) takes its potential and counting radii from pair[t_i][t_j]; a
 * type's valency f and shift delta come from its diagonal entry.  Particle i
 * counts neighbour j only if count_mask[t_i][t_j] is 1, so
 *   n_i = sum_{j: mask[t_i][t_j]} omega(r_ij; r_l^{ij}, r_h^{ij}),
 *   s_i = omega(n_i; f_{t_i} - delta_{t_i}, f_{t_i} - delta_{t_i} + 1),
 *   U   = sum_{i<j} [V_r^{ij} + s_i s_j V_a^{ij}] + sum_bonds k_bond/2 (r - r0_bond)^2.
 * Bonded pairs keep their non-bonded terms.  All arrays are host memory in
 * the caller's particle order, copied at creation; row-major tables. */
#define VBC_MAX_TYPES 8
typedef struct {
    int32_t ntypes;                /* 1 <= ntypes <= VBC_MAX_TYPES */
    const int32_t* type;           /* [n] type of each particle, in [0, ntypes) */
    const vbc_pair_params* pair;   /* [ntypes][ntypes], symmetric in r_r, r_a, r_l, r_h, E_r, E_a */
    const int32_t* count_mask;     /* [ntypes][ntypes] of 0 or 1: row type counts column type */
    int64_t nbonds;                /* bonds, >= 0 */
    const int64_t* bonds;          /* [nbonds][2] particle indices, i != j, each bond once (NULL if none) */
    double k_bond, r0_bond;        /* harmonic constant (>= 0) and rest length (>= 0) */
} vbc_types;

/*
 * Create a multi-type system.  cfg is as for vbc_create_system except that
 * cfg->params is ignored (the neighbour list reaches the largest
 * max(r_r, r_a, r_h) of the table plus the skin).  cfg->precision selects
 * the arithmetic as for one type: VBC_FP64, or VBC_FP32_SPLIT (cubic box;
 * exact fixed-point counts, FP32 pair and bond terms, FP64 state, energies
 * and virial).  Every other call then works on it as on any system, except
 * vbc_set_params and vbc_get_observables (INVALID_ARG).  Errors as
 * vbc_create_system, and INVALID_ARG for a bad type, table, mask or bond.
 */
int vbc_create_typed_system(const vbc_config* cfg, const vbc_types* types, vbc_system** out);

/* Device memory, in bytes, that vbc_create_system would allocate for cfg (the
 * initial capacities; the first list build trims them, an overflow grows
 * them).  No device is touched.  Errors: INVALID_ARG (NULL pointers, n, box or
 * skin out of range, box too small for the cell list). */
int vbc_estimate_device_bytes(const vbc_config* cfg, int64_t* bytes);

/* Force a neighbour-list rebuild now (Morton sort of the particles, cell list,
 * Verlet list of radius r_c + skin).  Rebuilds also happen automatically when a
 * particle has moved more than skin/2 since the last build. */
int vbc_build_neighbors(vbc_system* sys);

/*
 * One VBC force/energy evaluation at the current positions (Sec. 2: pass 1
 * counts, chain-rule pass, pass 2 forces).  Every output is optional (NULL):
 *   F      [n][3]  forces -grad U
 *   counts [n]     smoothed neighbour counts n_i (Eq. counter)
 *   energy [1]     U = sum_{i<j} V^(r_ij) (Eq. Vhat), accumulated in FP64
 *   virial [1]     W = sum_{i<j} (x_i - x_j) . F_ij, accumulated in FP64
 * outputs_on_device says whether the four pointers are device memory.
 */
int vbc_compute_forces(vbc_system* sys, double* F, double* counts, double* energy,
                       double* virial, int outputs_on_device);

/*
 * Per-particle intermediates of the last vbc_compute_forces, for diagnostics:
 * s [n] = omega(n_i; f - delta, f - delta + 1), ds [n] = ds/dn, A [n] = dU/dn_i.
 * Any pointer may be NULL.
 */
int vbc_get_switch(vbc_system* sys, double* s, double* ds, double* A, int outputs_on_device);

/*
 * The Verlet list of the last build, in caller order, for diagnostics:
 * nnb [n] list lengths (pairs within r_c + skin at build time), nbr [n][cap]
 * neighbour indices (the first min(nnb[i], cap) entries of row i are written).
 * Lists are complete (every pair closer than r_c + skin at the build) and
 * hold no pair at or beyond that radius.
 */
int vbc_get_neighbors(vbc_system* sys, int32_t* nnb, int32_t* nbr, int32_t cap, int outputs_on_device);

/*
 * Advance nsteps Langevin steps (BAOAB splitting, unit mass): half kick, half
 * drift, exact Ornstein-Uhlenbeck velocity update with c1 = exp(-gamma dt) and
 * noise sqrt((1 - c1^2) kT) xi, half drift, force evaluation, half kick.  The
 * three normals xi of particle id at step counter k come from
 * Philox4x32-10 (counter (k lo, k hi, id, 0), key (seed lo, seed hi)) through
 * Box-Muller on u = ((word >> 9) + 1/2) / 2^23.  Requires dt > 0, kT >= 0,
 * gamma >= 0.  Errors: UNSTABLE if a position or velocity becomes
 * non-finite (the state is then the one of the failing step).
 */
int vbc_step_langevin(vbc_system* sys, int64_t nsteps, double dt, double kT, double gamma);

/* Checkpoint: copy out unwrapped positions, velocities and the step counter
 * (any pointer may be NULL).  Restoring them with vbc_set_state resumes the
 * trajectory, the same one to rounding: sums follow the sorted layout the
 * system holds at the time.  vbc_set_state keeps the neighbour list when
 * every loaded position lies within skin / 2 of the position at the last
 * build (as the step loop does), and has it rebuilt by the next pass
 * otherwise, or when the system was halted.  A load clears every halt,
 * including the one a batched step that gave up (TIMEOUT) leaves.  Errors:
 * UNSTABLE for a non-finite or out-of-range value (the system then stays
 * halted until a good state is loaded). */
int vbc_get_state(vbc_system* sys, double* pos, double* vel, int64_t* step, int on_device);
int vbc_set_state(vbc_system* sys, const double* pos, const double* vel, int64_t step,
                  int on_device);

/* Change the pair parameters of an existing system (same cut-off or smaller:
 * r_c + skin must still fit the cell grid built at creation).  The neighbour
 * list is rebuilt before the next pass. */
int vbc_set_params(vbc_system* sys, const vbc_pair_params* params);

int vbc_get_stats(vbc_system* sys, vbc_stats* out);

/*
 * Thermodynamic reductions of the current state, all in FP64 with fixed-order
 * (deterministic) sums on the device:
 *   U         = sum_{i<j} [V_r(r_ij) + s_i s_j V_a(r_ij)]        Eq. (Vhat), Sec. 2
 *   W         = sum_{i<j} -g_ij r_ij, g_ij = dU/dr_ij with the chain-rule term (pair virial)
 *   KE        = sum_i |v_i|^2 / 2 (unit mass; kinetic temperature 2 KE / (3 N))
 *   mean_n    = (1/N) sum_i n_i, n_i of Eq. (counter) (masked counts for multi-type systems)
 *   in_window = particles with f - delta < n_i < f - delta + 1 (s'_i != 0), Eq. (Psidelta)
 *   pairs_within_rc = unordered pairs with r_ij < r_c
 *   step      = the step counter of the state
 * The counts, s, s' and A behind U, W, mean_n and in_window are recomputed in
 * FP64 from the state (U to 1e-9 relative of the FP64 definition).  The call
 * changes neither the state nor the forces the next vbc_step_langevin opens
 * with, so logging between chunks of steps leaves the trajectory bitwise the
 * same.  out is a host struct.  Errors: INVALID_ARG (NULL), CUDA, UNSTABLE
 * (halted system), NLIST_OVERFLOW.
 */
typedef struct {
    double U;
    double W;
    double KE;
    double mean_n;
    int64_t in_window;
    int64_t pairs_within_rc;
    int64_t step;
} vbc_thermo;
int vbc_compute_thermo(vbc_system* sys, vbc_thermo* out);

/*
 * Per-kernel timing with CUDA events on the system's stream.  enable != 0
 * starts recording one event pair around every kernel launch (up to
 * max_launches launches; further launches are not timed); enable == 0 stops.
 * vbc_profile_read synchronises the stream and returns, for kernel class
 * `which` (VBC_K_*), the summed device time in milliseconds and the number of
 * timed launches.
 */
enum { VBC_K_REBUILD = 0, VBC_K_COUNT = 1, VBC_K_CHAIN = 2, VBC_K_FORCE = 3, VBC_K_ENERGY = 4,
       VBC_K_NCLASSES = 5 };
int vbc_profile(vbc_system* sys, int enable, int64_t max_launches);
int vbc_profile_read(vbc_system* sys, int which, double* total_ms, int64_t* launches);

/* Number of kernel launches the library has issued (all kinds) since creation. */
int64_t vbc_kernel_launches(vbc_system* sys);

/*
 * Force evaluation that allocates nothing (the paper has no counterpart: this
 * is a deployment aid).  Some callers cannot call cudaMalloc -- code running
 * under another framework's allocator or fixed memory budget, real-time loops
 * that must not pay an allocation's latency or risk its failure, plug-ins that
 * are handed device buffers but may not create their own.  This call needs no
 * vbc_system: it evaluates the counts and forces of one small system with the
 * same FP32-split arithmetic as vbc_compute_forces (all pairs instead of a
 * neighbour list), keeping the scratch that its passes exchange in one
 * file-scope device array of VBC_NOALLOC_MAX_N * 28 bytes (448 KiB).  Every
 * GPU that loads the library holds that array until the process exits.
 *
 *   n       1 <= n <= VBC_NOALLOC_MAX_N (larger n returns VBC_ERR_INVALID_ARG)
 *   box     [3] host array, a cube of edge >= 2 max(r_r, r_a, r_h)
 *   pos     [n][3] device array of positions (any periodic image)
 *   params  host pointer to the pair parameters
 *   F       [n][3] device array, receives the forces
 *   counts  [n] device array for n_i, or NULL
 *   stream  cudaStream_t to run on (NULL = default stream); returns after it finishes
 *
 * The first call on a device looks up the device address of the scratch array
 * (once per device, with that device current); make that first call before any
 * stream capture.  Calls never call cudaMalloc, cudaFree or an allocating
 * library routine.  All calls share the one array: each call writes every
 * scratch entry it reads, so nothing carries over from a previous call, but
 * calls whose work overlaps on the GPU (two streams, two host threads) race
 * with each other and must be serialised by the caller.
 */
#define VBC_NOALLOC_MAX_N 16384
int vbc_compute_forces_noalloc(int32_t n, const double* box, const double* pos, const vbc_pair_params* params,
                               double* F, double* counts, void* stream);

/* Release everything the system owns.  NULL is accepted. */
void vbc_destroy(vbc_system* sys);

/* Message describing the last error of the calling thread ("" if none). */
const char* vbc_last_error(void);

/* ------------------------------------------------------------------ batched stepping
 * Many independent systems of uneven size (parameter sweeps, Sec. 5) advanced
 * together on one GPU.  vbc_batch_step runs each system's Langevin iterations
 * exactly as vbc_step_langevin does; the systems' two-step graphs are
 * captured side by side into one CUDA graph, so that one graph launch
 * advances every system by two steps and the small systems' kernels fill the
 * GPU together.  The first and last iterations run on each system's own
 * stream, and a system whose neighbour list overflows is grown and finishes
 * its iterations on its own.  The results are bitwise those of stepping each
 * system alone.  The systems stay owned by the caller and must outlive the
 * batch; they must share one device and appear once each. */
typedef struct vbc_batch vbc_batch;

/* Errors: INVALID_ARG (NULL or repeated systems, count < 1, systems on
 * different devices), CUDA. */
int vbc_batch_create(vbc_system* const* systems, int32_t count, vbc_batch** out);

/* Advance every system of the batch by nsteps steps, as vbc_step_langevin
 * does, system k at temperature kT[k] ([count] host array); dt and gamma are
 * shared.  Returns the first error of any system; the others are advanced all
 * the same. */
int vbc_batch_step(vbc_batch* batch, int64_t nsteps, double dt, const double* kT, double gamma);

/* Release the batch (not its systems).  NULL-safe. */
void vbc_batch_destroy(vbc_batch* batch);

/*
 * How a batch advances (the paper has no counterpart; its parameter sweeps of
 * Sec. 5 motivate running many systems on one GPU).  VBC_BATCH_FUSED (the
 * default): iteration 0 of each system on its own stream, then one
 * cooperative launch per Langevin iteration for all systems together, whose
 * phases (gate, list rebuilds, counts, chain-rule terms, forces, update) take
 * the work items of every system and are separated by grid-wide waits; the
 * result of each system is bitwise the one it gets stepped alone.  It takes
 * single-type systems of one precision on the default row-walk block shape;
 * any other batch, or one whose largest system does not fit the launch's
 * shared memory, runs as VBC_BATCH_GRAPHS: each system's two-step graph
 * captured side by side into one CUDA graph.
 * wait_limit: spins (of about 100 ns each) a grid-wide wait makes before it
 * gives up; < 0 restores the default (2^22, about half a second).  A wait that
 * gives up ends the launch: vbc_batch_step then returns VBC_ERR_TIMEOUT and
 * every system of the batch is halted (its state incomplete) until
 * vbc_set_state loads a state again; the GPU context stays usable.
 * Errors: INVALID_ARG.
 */
enum { VBC_BATCH_FUSED = 0, VBC_BATCH_GRAPHS = 1 };
int vbc_batch_set_mode(vbc_batch* batch, int mode, int64_t wait_limit);

/* Fused launches the batch has issued (one per iteration of vbc_batch_step). */
int64_t vbc_batch_fused_launches(vbc_batch* batch);

/* ------------------------------------------------------------------ autotuning
 * The close-neighbour count and the row walks run resident grids, as many
 * blocks per SM as fit by default.  For small systems (and many systems side
 * by side, as in batches and serving) fewer blocks can be faster, and dense
 * walks (most particles unsaturated) can gain from larger blocks, which give
 * each row more threads.  The grid sizes change no result: every row and
 * every cell group is computed the same way whichever block takes it.  The
 * block shape and the threads-per-row cap decide how a dense walk splits a
 * row between threads, and so the order of its floating-point sums: they
 * change forces, chain-rule terms and FP64 counts by rounding only (the
 * FP32-split counts, integer sums, not at all), and every setting is
 * deterministic. */
typedef struct {
    int32_t rows_blocks_per_sm;     /* the row walks' grid, 0 = as many as fit */
    int32_t count_blocks_per_sm;    /* the close-neighbour count's grid, 0 = as many as fit */
    int32_t rows_threads_per_block; /* the row walks' block shape: 128, 256 or 512 (0 = 128) */
    int32_t threads_per_row_max;    /* threads per row of a dense walk, at most: 1, 2, 4, ..., 32 (0 = 32) */
    double ms_per_step;             /* the best trial's time per step (vbc_autotune's output) */
} vbc_tuning;

/* Apply grid settings (for example the result of an earlier vbc_autotune on a
 * system of the same shape).  ms_per_step is ignored.  Errors: INVALID_ARG. */
int vbc_set_tuning(vbc_system* s, const vbc_tuning* t);

/* Time trial_steps Langevin steps (dt, kT, gamma as vbc_step_langevin) for
 * each candidate setting, one knob at a time (block shape, row grid, threads
 * per row, count grid), keep the fastest and return it (the default stays
 * unless a setting beats it by 2%).  The trials advance the system (about
 * 14 (trial_steps + 2) steps).  Errors: INVALID_ARG (NULL out, trial_steps
 * < 4), as vbc_step_langevin otherwise. */
int vbc_autotune(vbc_system* s, int64_t trial_steps, double dt, double kT, double gamma, vbc_tuning* out);

/* ------------------------------------------------------------------ observables
 * Valency observables of Sec. 3 on the current state: two particles are
 * neighbours when r_ij < r_a (strict; an instantaneous distance criterion, so
 * transient contacts count as well as bonds).  z_i is the number of
 * neighbours of particle i, <z> its mean, and P_err the fraction of particles
 * with z_i > f (over-coordination).  Integer sums on the device, so the
 * figures do not depend on the launch. */
#define VBC_ZHIST 32
typedef struct {
    double mean_z;                /* <z> */
    double p_err;                 /* fraction of particles with z_i > f */
    int64_t z_hist[VBC_ZHIST];    /* particles with z_i = k; the last bin holds z_i >= VBC_ZHIST - 1 */
} vbc_observables;

/* Fill *out; if z is not NULL, also z_i per particle ([n] int32, caller's
 * particle order; a device pointer if on_device).  Rebuilds the neighbour
 * list first if it is due.  Errors: INVALID_ARG (NULL out), CUDA, OOM,
 * NLIST_OVERFLOW. */
int vbc_get_observables(vbc_system* s, vbc_observables* out, int32_t* z, int on_device);

/* ------------------------------------------------------------------ serving
 * Many independent simulations (valency and temperature sweeps, Sec. 5: one
 * system per parameter set) on one GPU.  A server admits submitted requests
 * in arrival order whenever a slot is free and the device memory of the
 * admitted systems, estimated by vbc_estimate_device_bytes and then taken
 * from each live system, stays within the budget.  Each slot is a host thread
 * with its own CUDA stream: it creates the request's system there, advances
 * it in chunks of chunk_steps Langevin steps with the state resident on the
 * device, copies the final state to host memory the server owns and
 * releases the system.  Requests that arrive while others run are admitted
 * as slots and memory free up, and the slots' kernels overlap on the device.
 * A system's result does not depend on what else runs: every kernel of the
 * library is deterministic and a system shares no device memory with
 * another, so a request alone and in a mix gives bitwise the same state. */
typedef struct vbc_server vbc_server;

typedef struct {
    int64_t hbm_budget;   /* device bytes the admitted systems may hold together (> 0) */
    int32_t slots;        /* systems advanced at the same time, 1 <= slots <= 256 */
    int64_t chunk_steps;  /* Langevin steps per chunk (> 0) */
} vbc_server_config;

typedef struct {
    vbc_config system;    /* as for vbc_create_system, host input only: stream and
                             inputs_on_device are ignored; pos and vel are copied at submit */
    int64_t nsteps;       /* Langevin steps to run (>= 0) */
    double dt, kT, gamma; /* as for vbc_step_langevin */
} vbc_request;

enum { VBC_REQ_QUEUED = 1, VBC_REQ_RUNNING = 2 };

typedef struct {
    int32_t status;       /* VBC_REQ_QUEUED, VBC_REQ_RUNNING, then VBC_OK or the error code */
    int64_t n;            /* particles */
    int64_t steps_done;   /* Langevin steps completed so far */
    double t_submit;      /* seconds on the server's clock (steady, from its creation) */
    double t_admit;       /* when a slot took it (0 while queued) */
    double t_done;        /* when its state was on the host (0 until then) */
    int64_t device_bytes; /* device memory reserved for it (estimate, then the live figure) */
} vbc_request_info;

/* Start a server: its slot threads wait for work.  Errors: INVALID_ARG, CUDA
 * (no device). */
int vbc_server_create(const vbc_server_config* cfg, vbc_server** out);

/* Queue a request; *id names it from here on.  The inputs are validated and
 * copied before the call returns; the work runs later on a slot.  Errors:
 * INVALID_ARG (as vbc_create_system, or a step argument out of range), OOM
 * (the estimate alone exceeds the budget). */
int vbc_server_submit(vbc_server* srv, const vbc_request* req, int64_t* id);

/* Wait up to timeout_s seconds (< 0: without limit) for request id to finish;
 * id = -1 waits for every request submitted so far.  Fills *info (may be
 * NULL; not for id = -1).  Returns VBC_OK when finished (the request's own
 * outcome is info->status), VBC_ERR_TIMEOUT if not finished in time,
 * INVALID_ARG for an unknown id. */
int vbc_server_wait(vbc_server* srv, int64_t id, double timeout_s, vbc_request_info* info);

/* Status of request id without waiting.  Errors: INVALID_ARG (unknown id). */
int vbc_server_info(vbc_server* srv, int64_t id, vbc_request_info* info);

/* Copy a finished request's final state ([n][3] positions, unwrapped, and
 * velocities, in the submitted particle order; either may be NULL) to host
 * memory and forget the request.  Errors: INVALID_ARG (unknown id, or not
 * finished yet), or the request's own error code (its state is then not
 * copied, and the request is forgotten all the same). */
int vbc_server_result(vbc_server* srv, int64_t id, double* pos, double* vel, vbc_request_info* info);

/* Stop the server: queued requests are dropped and running ones stop after
 * their current chunk (both end with status VBC_ERR_CANCELLED), the slot
 * threads end, and everything is released.  NULL-safe. */
void vbc_server_destroy(vbc_server* srv);

/* Message of the last failed vbc_server_* call on this thread (a request's own
 * failure reads back through vbc_server_result). */
const char* vbc_server_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VBC_H */
