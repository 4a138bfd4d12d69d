/*
 * ljmd.h -- C ABI of the GB300 truncated Lennard-Jones MD library (libljmd.so).
 *
 * The library advances N particles in a periodic orthorhombic box under
 * truncated(-shifted) Lennard-Jones pair forces with the velocity-Verlet
 * integrator, using Verlet neighbour lists built by particle binning -- the
 * MD hot path of arXiv 2406.04210 (Sec. 3, Code structure: modules for
 * forces and integrators, `integrate`/`finalize` half steps around the
 * `force` evaluation, Verlet lists from a spatial decomposition; Sec. 4:
 * Lennard-Jones pair forces with velocity-Verlet; Sec. 5, Truncated Force
 * Performance Study: truncated pair forces over Verlet lists, whose force and
 * list-update kernels dominate the run time).  The paper gives the problem,
 * not formulas; the textbook forms used are:
 *
 *   U_ab(r) = 4 eps_ab [(sigma_ab/r)^12 - (sigma_ab/r)^6] - shift_ab, r < rc_ab
 *   F_i = sum_{j != i, r_ij < rc} 48 eps/r^2 [(sigma/r)^12 - (sigma/r)^6/2] d_ij,
 *         d_ij = minimum image of x_i - x_j
 *   integrate: v += dt/2 F; x += dt v     (unit mass)
 *   finalize:  v += dt/2 F
 *   E_pot = sum_{i<j} U, W = sum_{i<j} d_ij . F_ij, E_kin = 1/2 sum v^2,
 *   T = 2 E_kin / (3N - 3)
 *
 * Conventions shared by every entry point
 *  - Array arguments are plain pointers that may point to host memory or to
 *    device memory of the machine's GPU; the library detects which
 *    (cudaPointerGetAttributes) and copies as needed.  Particle arrays are in
 *    USER order (the order given at creation), n x 3 row-major (AoS) FP64
 *    unless stated.  The library never keeps a caller pointer after a call
 *    returns.
 *  - Calls are ordered after work already queued on the `stream` given at
 *    creation, and work queued on that stream afterwards is ordered after the
 *    call.  Calls return once their results are in the caller's buffers
 *    (every call synchronises the box's internal stream before returning).
 *  - Errors are returned as md_status; nothing is thrown across the ABI.  A
 *    message for the last failing call of a box is in md_last_error().
 *  - A box (md_box) owns all of its device memory.  Memory comes from the
 *    allocator installed with md_set_allocator (default: cudaMalloc/cudaFree).
 *  - A batch holds nrep independent replicas (boxes of their own, each with
 *    its own particle count and edge lengths, sharing the LJ parameters); a
 *    single box is a batch with nrep = 1.  Batched arrays concatenate the
 *    replicas in order.
 */
#ifndef LJMD_H
#define LJMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_box md_box;

typedef enum {
    MD_OK = 0,
    MD_ERR_ARG = 1,            /* invalid argument or call order                */
    MD_ERR_CUDA = 2,           /* a CUDA runtime call failed                    */
    MD_ERR_OOM = 3,            /* the allocator returned NULL                   */
    MD_ERR_CAPACITY = 4,       /* neighbour-list capacity exceeded (the library
                                  regrows and retries internally; returned only
                                  if the regrow itself fails)                   */
    MD_ERR_BOX_TOO_SMALL = 5,  /* rc_max + skin >= half a box edge             */
    MD_ERR_NONFINITE = 6,      /* a non-finite force or position was produced   */
    MD_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up            */
    MD_ERR_STATE = 8           /* no matching forward record (md_adjoint)       */
} md_status;

/* Arithmetic of a box (Sec. 3, Code structure: modules carry a floating-point
 * type "single, mixed precision, double"; the mixed form is HAL's MD
 * double-single accumulation). */
typedef enum {
    MD_PREC_MIXED_DS = 0,   /* FP32 pair forces from cell-relative offsets,
                               double-single (2 x FP32) positions/velocities   */
    MD_PREC_MIXED_FP64 = 1, /* FP32 pair forces, FP64 positions/velocities     */
    MD_PREC_FP64 = 2        /* FP64 pair forces and FP64 integration           */
} md_precision;

/* Device allocator hook (no counterpart in the paper: memory plumbing for
 * hosts such as PyTorch that pool device memory): alloc(bytes, ctx) returns a
 * device pointer of the current device aligned to 256 bytes, or NULL;
 * free(ptr, ctx) releases it.
 * Installed process-wide; boxes created afterwards use it for every device
 * allocation they make (at creation, md_set_lj and list regrowth).  Passing
 * NULL functions restores cudaMalloc/cudaFree.  Not thread-safe against
 * concurrent box creation. */
typedef void* (*md_alloc_fn)(size_t bytes, void* ctx);
typedef void (*md_free_fn)(void* ptr, void* ctx);
md_status md_set_allocator(md_alloc_fn alloc, md_free_fn free_, void* ctx);

/* Create a batch of nrep replicas on the current CUDA device (Sec. 1 and
 * Sec. 3: N particles in a periodic box; the replicas are independent
 * systems of that kind).
 *   n[nrep]        particle count of each replica (>= 0)
 *   box[nrep*3]    edge lengths (Lx, Ly, Lz) of each replica (> 0)
 *   type[sum n]    species id of each particle (0 <= type < ntypes given to
 *                  md_set_lj), or NULL for all zero
 *   pos[sum n * 3] positions; any real values (wrapped into [0, L) on entry)
 *   vel[sum n * 3] velocities, or NULL for zero
 *   stream         cudaStream_t the calls are ordered with (NULL = legacy)
 * Host-array arguments n and box must be host memory.  md_set_lj must be
 * called before any force, update or integrate call. */
md_status md_batch_create(md_box** out, int32_t nrep, const int64_t* n,
                          const double* box, const int32_t* type,
                          const double* pos, const double* vel,
                          md_precision prec, void* stream);

/* md_batch_create with nrep = 1; box[3] is host memory.  Both copy the
 * inputs (the caller keeps ownership of its arrays) and return MD_ERR_ARG
 * for out == NULL, nrep < 1, a negative n, a non-positive or non-finite
 * edge, pos == NULL with particles, or more than 2^26 particle slots,
 * MD_ERR_OOM when the allocator fails and MD_ERR_CUDA when a CUDA call
 * fails. */
md_status md_box_create(md_box** out, int64_t n, const double box[3],
                        const int32_t* type, const double* pos,
                        const double* vel, md_precision prec, void* stream);

/* Free all device memory of the box (after its queued work completes) and
 * the box itself; MD_ERR_ARG for NULL. */
md_status md_box_destroy(md_box* b);

/* Set the truncated LJ pair parameters (host arrays, ntypes x ntypes,
 * row-major, symmetric; 1 <= ntypes <= 8), the Verlet skin and whether the
 * energy is shifted to zero at the cutoff.  The list radius is
 * rl = max(rcut) + skin; cells are floor(L/rl) per dimension.  Returns
 * MD_ERR_BOX_TOO_SMALL if rl >= L/2 for any replica.  Rebuilds the lists and
 * recomputes the forces at the current positions.
 * All-pairs form (Sec. 4: the untruncated LJ interaction between all
 * particles): every rcut = +INFINITY.  Forces then sum over every pair of a
 * replica with the minimum image and no lists; the skin only sets how often
 * positions are re-wrapped.  md_adjoint, md_pair_hist, md_get_nlist and
 * md_autotune return MD_ERR_ARG in this form. */
md_status md_set_lj(md_box* b, int32_t ntypes, const double* eps,
                    const double* sigma, const double* rcut, double skin,
                    int32_t energy_shift);

/* Stochastic Andersen-like thermostat (Sec. 4: the "Boltzmann" thermostat of
 * the all-to-all workload).  After the finalize half kick of every step of
 * md_integrate, each particle collides with the heat bath with probability
 * rate * dt; its velocity is then redrawn from the Maxwell-Boltzmann
 * distribution at T_bath[r] of its replica (unit mass).  The random numbers
 * are Philox4x32-10 (Salmon et al., SC'11) with key = seed + replica index
 * and counter = (index of the particle inside its replica, step index low,
 * step index high, 0 or 1); the step index counts the steps since this call.
 * Word 0 decides the collision (below floor(rate dt 2^32)); the three
 * Gaussians come by Box-Muller from words 1,
 * 2 and from words 0, 1 of the second counter.  Energies are taken after
 * the collisions.  rate = 0 switches it off (the default: NVE).
 *   T_bath  host, nrep entries (> 0), or NULL with rate = 0
 * md_integrate with ckpt_every > 0 returns MD_ERR_ARG while it is on (the
 * reverse of a stochastic collision is not defined). */
md_status md_set_thermostat(md_box* b, const double* T_bath, double rate,
                            uint64_t seed);

/* Neighbour-list update (Sec. 3, Code structure; Sec. 5): re-bin and rebuild
 * the lists of every replica in which some particle moved more than skin/2
 * since its last build, or of all replicas if force_rebuild != 0.  *rebuilt
 * (nullable, host) receives the number of replicas rebuilt. */
md_status md_neighbour_update(md_box* b, int32_t force_rebuild,
                              int32_t* rebuilt);

/* Pair forces, potential energy and virial at the current positions (Sec.
 * 4: the Lennard-Jones pair force; Sec. 5, Truncated Force Performance
 * Study: truncated forces over the Verlet lists), updating the lists first
 * if the skin rule asks.
 *   force_out  nullable, (sum n) x 3 FP64, user order, host or device
 *   epot, virial nullable, nrep entries each (E_pot and W per replica), host
 *              or device
 * Returns MD_ERR_ARG before md_set_lj, MD_ERR_NONFINITE for a non-finite
 * force, MD_ERR_TIMEOUT if a bounded device wait gave up. */
md_status md_force(md_box* b, double* force_out, double* epot, double* virial);

/* Advance nsteps velocity-Verlet steps of size dt (Sec. 3, Fig. 1:
 * integrate, force, finalize; Sec. 4: velocity-Verlet), rebuilding lists by
 * the skin rule (Sec. 3; Sec. 5: the list update).  The steps run as CUDA
 * graphs of up to 100 steps each, captured on first use.
 *   ckpt_every  0: plain run.  k > 0: record the run for md_adjoint, storing
 *               the state every k steps (nsteps must be a multiple of k).
 *   thermo_out  nullable, nsteps x nrep x 4 FP64: E_pot, E_kin, W, T after
 *               each step.  When NULL no energies are computed. */
md_status md_integrate(md_box* b, double dt, int64_t nsteps, int32_t ckpt_every,
                       double* thermo_out);

/* Reverse-mode derivative of the run recorded by the last md_integrate with
 * ckpt_every > 0 (its checkpoints are replayed segment by segment).
 *   lam_x_T, lam_v_T  dL/dx and dL/dv at the end of the run, (sum n) x 3
 *   lam_x_0, lam_v_0  out: dL/dx_0 and dL/dv_0, (sum n) x 3
 *   dL_deps, dL_dsigma out (nullable): ntypes x ntypes, symmetric; the entry
 *                     (a,b) is the derivative with respect to the single
 *                     symmetric parameter eps_ab (sigma_ab), rcut held fixed.
 * The paper has no adjoint; this follows from differentiating the steps
 * above (velocity-Verlet is differentiated exactly, one Hessian-vector
 * product of U per step, evaluated in FP32 with the recorded lists; the
 * adjoint state is FP64).  Each segment of ckpt_every steps is replayed from
 * its checkpoint bit for bit (a recorded run rebuilds the lists at every
 * checkpoint).  Returns MD_ERR_STATE if no recorded run exists (recording is
 * dropped by md_set_lj and md_set_state).  The box's state after the call is
 * the end-of-run state.  Batched boxes return parameter gradients summed
 * over replicas (the parameters are shared). */
md_status md_adjoint(md_box* b, const double* lam_x_T, const double* lam_v_T,
                     double* lam_x_0, double* lam_v_0, double* dL_deps,
                     double* dL_dsigma);

/* Smoothed pair-distance histogram of the current positions and its
 * gradient, a trajectory loss for md_adjoint (no counterpart in the paper):
 *   h[r, k] = (1/n_r) sum_{i<j in replica r, r_ij < rmax} exp(-(r_ij - c_k)^2 / (2 width^2)),
 *   c_k = (k + 1/2) rhist / nbins,  k = 0 .. nbins-1  (1 <= nbins <= 256)
 *   hist  nullable, nrep x nbins FP64 out
 *   coef  nullable, nrep x nbins FP64: with grad, grad receives
 *         d/dx sum_{r,k} coef[r,k] h[r,k], (sum n) x 3 FP64, user order
 * rmax must not exceed the list radius (rcut + skin); the lists are rebuilt
 * first if the particles moved since the last build.  Distances are FP32. */
md_status md_pair_hist(md_box* b, int32_t nbins, double rhist, double width,
                       double rmax, const double* coef, double* hist,
                       double* grad);

/* md_force without any allocation (the paper has no counterpart; this serves
 * library users).  Some callers cannot allocate device memory when they need
 * forces: a framework that owns all GPU memory through its own pool, a pool
 * that is capped or frozen, or a loop that must not block in an allocator.
 * md_force may grow box-owned buffers on first use; this call never
 * allocates, on the device or through the allocator hook.  Its scratch (the
 * per-128-particle energy/virial partial sums and the per-replica totals) is
 * a static device array of 524,288 doubles (4 MiB) that every GPU loading
 * the library holds until the process exits; boxes needing more (16 doubles
 * per 128 particles with FP32 forces, 8 all-FP64, 2 in the all-pairs form,
 * + 4 per replica; about 4.19M particles for one box) are rejected with
 * MD_ERR_ARG and a message.  The first call on a device looks up that array's address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array and overwrite what they use, so calls whose
 * GPU work overlaps (on different streams or boxes) race.
 *   force_out  nullable; DEVICE memory, (sum n) x 3 FP64, user order
 *   epot, virial nullable, nrep entries each, host or device
 * The lists must be current (as after md_set_lj, md_integrate or
 * md_neighbour_update); results equal md_force's. */
md_status md_force_noalloc(md_box* b, double* force_out, double* epot,
                           double* virial);

/* Current state in user order (no counterpart in the paper: state access):
 * pos in [0, L) FP64, vel FP64, image counts (number of box lengths crossed),
 * each nullable, host or device, (sum n) x 3. */
md_status md_get_state(md_box* b, double* pos, double* vel, int32_t* image);

/* Replace positions (wrapped into [0,L)) and, if vel != NULL, velocities
 * (no counterpart in the paper: state access); image counts are reset to
 * zero; lists are rebuilt and forces recomputed; MD_ERR_ARG for a NULL pos
 * with particles. */
md_status md_set_state(md_box* b, const double* pos, const double* vel);

/* Neighbour lists as last built, for inspection (Sec. 3: the Verlet lists;
 * the call itself has no counterpart in the paper): count[sum n] (user order)
 * and, if nbr != NULL, the user indices of each particle's neighbours in
 * nbr[i*cap ...] (unsorted; entries beyond count are left untouched); pos
 * (nullable) receives the FP64 positions the lists were built from.  Returns
 * MD_ERR_CAPACITY if some count exceeds cap (counts are still written). */
md_status md_get_nlist(md_box* b, int32_t* count, int64_t* nbr, int64_t cap,
                       double* pos);

typedef struct {
    int64_t n_total;        /* sum of n over replicas                         */
    int32_t nrep;
    int32_t ntypes;
    int32_t capacity;       /* neighbour-list slots per particle              */
    int32_t precision;      /* md_precision                                   */
    int64_t ncell_total;    /* cells over all replicas                        */
    int64_t rebuilds;       /* list builds so far (summed over replicas)      */
    int64_t steps;          /* velocity-Verlet steps done                     */
    int64_t device_bytes;   /* device memory held                             */
    double rlist;           /* max(rcut) + skin                               */
    int64_t launches;       /* kernels launched so far (graph nodes included) */
    int64_t list_entries;   /* sum of list lengths at the last builds          */
    int64_t record_id;      /* serial number of the recorded forward run that
                               md_adjoint would differentiate now: each
                               md_integrate with ckpt_every > 0 takes the next
                               number; 0 when no record is valid (any call that
                               changes the state or the parameters drops it) */
} md_info;

md_status md_get_info(md_box* b, md_info* out);

/* Launch and layout tuning (Sec. 3 and Sec. 5: the paper determines launch
 * configurations per device; here they are set or timed per box), t[4]:
 *   t[0] blocks per SM of the pair-force kernels  (0 = default: 6, FP64 12)
 *   t[1] blocks per SM of the list build          (0 = default: 6)
 *   t[2] cells per list-build segment, <= 16      (0 = automatic: ~1400
 *        particles per 27-cell tile)
 *   t[3] neighbour-list slots per particle       (0 = automatic: fitted to
 *        1.1 x the longest list + 8 after the first build); always rounded
 *        up to a multiple of 16 (the FP32 force kernel reads 16-entry blocks)
 * Lists always regrow by themselves when a build needs more slots.
 * md_set_tuning applies t now (rebuilding the lists if t[2] or t[3] asks);
 * md_get_tuning reads the current values. */
md_status md_set_tuning(md_box* b, const int32_t t[4]);
md_status md_get_tuning(md_box* b, int32_t t[4]);

/* Cell layout, the binning's part of the tuning (Sec. 3: Verlet lists from a
 * spatial decomposition, "particle binning"; particles sorted for
 * locality):
 *   cell_scale  cell edge over the list radius, >= 1 (default 1: the most
 *               cells the 27-cell stencil allows, floor(L / rl) per
 *               dimension; larger values give fewer, fuller cells)
 *   order       order of the particles inside a cell: MD_ORDER_ZRUN (0,
 *               default) by z offset from the cell centre, which lets the
 *               list build take only the run of each neighbour cell within
 *               reach along z; MD_ORDER_MORTON (1) by a space-filling (Morton)
 *               curve over the cell's 4 x 4 x 4 sub-cells, then z, for
 *               locality of the neighbour gathers (the list build then scans
 *               whole neighbour cells)
 * md_set_layout re-bins the particles and rebuilds the lists when either
 * changes (results are unchanged up to FP32 summation order; the lists are
 * the same sets).  Not in the all-pairs form (one cell per replica). */
enum { MD_ORDER_ZRUN = 0, MD_ORDER_MORTON = 1 };
md_status md_set_layout(md_box* b, double cell_scale, int32_t order);
md_status md_get_layout(md_box* b, double* cell_scale, int32_t* order);

/* List-build kernel (Sec. 3: Verlet lists from the cell decomposition; the
 * lists are the same sets either way, decided exactly as the FP64
 * definition |d_ij|^2 < rl^2):
 *   MD_LIST_QUADS  one block per segment of cells, the segment's 27-cell
 *                  neighbourhood staged in shared memory, each warp taking
 *                  quads of particles with the candidates spread over its
 *                  lanes (each neighbour cell narrowed to its z-run within
 *                  reach under MD_ORDER_ZRUN)
 *   MD_LIST_LANES  one warp per cell, one lane per particle of the cell; the
 *                  warp stages each candidate once (dropping those beyond
 *                  the list radius of the cell's box) and every lane tests
 *                  it against its own particle; each lane's row is buffered
 *                  in shared memory as 16-bit codes (48 per lane) and
 *                  written out in 16-entry blocks
 *   MD_LIST_AUTO   (default) MD_LIST_LANES
 * The setting takes effect at the next list build. */
enum { MD_LIST_AUTO = 0, MD_LIST_QUADS = 1, MD_LIST_LANES = 2 };
md_status md_set_list_kernel(md_box* b, int32_t kind);
md_status md_get_list_kernel(md_box* b, int32_t* kind);

/* FP32 pair-force kernel of the list form (Sec. 4/5: LJ pair forces over the
 * Verlet lists; Sec. 5 finds that kernel bound by fetching neighbour data).
 * Both give the forces, energy and virial of the same lists, equal up to
 * FP32 rounding:
 *   MD_FORCE_CHUNKS  work items of 128 consecutive particles, 4 threads per
 *                    particle, neighbour offsets gathered from global memory
 *                    through L1, the image shift decoded from each entry
 *   MD_FORCE_TILES   work items of up to 2 x 2 x 2 cells ("bricks"): a
 *                    producer warp stages the next brick's neighbourhood (up
 *                    to 4 x 4 x 4 cells, at most 2048 particles) into shared
 *                    memory in the frame of the brick's centre while eight
 *                    consumer warps compute the current one, 4 threads per
 *                    particle, two pairs at a time in FP32-pair arithmetic;
 *                    a brick with a larger neighbourhood is evaluated from
 *                    global memory; device waits are bounded (a timeout is
 *                    reported as MD_ERR_TIMEOUT by the call)
 *   MD_FORCE_AUTO    (default) MD_FORCE_CHUNKS until md_autotune times both
 *                    and sets the faster one
 * On the 4M-particle fluid the chunk kernel is the faster (0.54 against
 * 0.65 ms per launch on GB300).  The FP64 precision and the all-pairs form
 * have kernels of their own and ignore the setting.  md_force_noalloc always
 * uses MD_FORCE_CHUNKS.  The setting takes effect at the next force
 * evaluation (the box's step graphs are re-captured); MD_ERR_ARG for another
 * kind, and md_get_force_kernel returns MD_ERR_ARG for a null pointer. */
enum { MD_FORCE_AUTO = 0, MD_FORCE_CHUNKS = 1, MD_FORCE_TILES = 2 };
md_status md_set_force_kernel(md_box* b, int32_t kind);
md_status md_get_force_kernel(md_box* b, int32_t* kind);

/* Step graphs: with on = 1 the list update of each captured step is a
 * conditional (IF) node, so steps without a list build launch one tiny kernel
 * instead of the rebuild sequence; with on = 0 (default) the rebuild kernels
 * are captured unconditionally and exit early when no build is due.  Results
 * are the same bit for bit.  On GB300 the node costs ~4.5 us per step more
 * than the early exits (measured at N = 2,000 and 97,556), so it pays only
 * in launch count.  Profilers cannot look inside graphs with conditional
 * nodes.  If the runtime refuses the node the box falls back to on = 0 by
 * itself; md_get_graph_conditional reads the mode in use. */
md_status md_set_graph_conditional(md_box* b, int32_t on);
md_status md_get_graph_conditional(md_box* b, int32_t* on);

/* Autotuner: times `reps` launches of the pair-force kernel for each
 * blocks-per-SM candidate, and `reps` forced list builds for each segment
 * length (automatic choice +-2) x list blocks-per-SM candidate, at the
 * current positions; applies the fastest and returns it in t[4] (as
 * md_get_tuning).  It then times the cell layouts (cell_scale 1, 1.08, 1.15 and 1.22,
 * each in both orders) as a step's cost -- one force evaluation plus a list
 * build spread over the box's observed steps per build (10 before any
 * step) -- and keeps the cheapest (md_get_layout reads it).  With the list
 * kernel on MD_LIST_AUTO it times both list kernels over the layouts and
 * sets the cheaper one (md_get_list_kernel reads it); a kernel set by
 * md_set_list_kernel is kept.  Then it times the list build's blocks per SM
 * again at the chosen layout and kernel.  Last, with the force kernel on
 * MD_FORCE_AUTO, it times both FP32 force kernels and sets the faster one
 * (md_get_force_kernel reads it).  The box's state is unchanged apart
 * from a list rebuild. */
md_status md_autotune(md_box* b, int32_t reps, int32_t t[4]);

/* Phase timing of md_integrate.  md_set_profiling(b, 1) resets the counters
 * and makes later md_integrate calls record CUDA events around each phase of
 * every step on the box's stream (inside the captured graphs); off by
 * default.  md_get_profile fills ms[4] (accumulated milliseconds) and
 * launches[4] (phase executions) for the phases 0 = integrate/finalize,
 * 1 = list update (binning, sort, list build; early exits included),
 * 2 = pair force, 3 = energy reductions.  Either output may be NULL. */
md_status md_set_profiling(md_box* b, int32_t on);
md_status md_get_profile(md_box* b, double* ms, int64_t* launches);

const char* md_last_error(const md_box* b);
const char* md_status_string(md_status s);

#ifdef __cplusplus
}
#endif

#endif /* LJMD_H */
