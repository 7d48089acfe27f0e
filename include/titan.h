/*
 * titan.h -- C ABI of the GB300 spring-mass simulator (libtitan.so).
 *
 * The library simulates the hot path of Titan (Austin et al., arXiv
 * 1911.10274): every time step applies each spring's Hooke-plus-damping force
 * to both of its masses (Sec. III-B, Eq. 1), then integrates every mass with
 * a velocity-first Euler step under gravity, a ground plane with Coulomb
 * friction, and fixed-mass constraints (Sec. III-A).  The host calls follow the
 * paper's asynchronous model (Sec. III-D): the caller builds the objects, lets
 * the GPU run a number of steps without blocking, reads state back without
 * stalling the step loop, edits the system between steps and resumes.
 *
 * Conventions for every call:
 *  - Pointers are host pointers unless the name says "dev".  Input arrays are
 *    owned by the caller and are copied before the call returns; the library
 *    keeps no pointer to them.
 *  - Mass and spring indices are always the caller's own (input) order; any
 *    internal reordering is invisible at this interface.
 *  - Every call returns a titan_status and never throws or aborts.  On an
 *    error the handle is unchanged unless the status is TITAN_E_CUDA, and
 *    titan_last_error() describes it.  Errors of earlier asynchronous GPU work
 *    are reported by the next call that synchronises with it.
 *  - Calls on one handle must not overlap; a call that finds another one in
 *    progress on the same handle returns TITAN_E_BUSY.  Distinct handles are
 *    independent and may be driven from different threads.
 *  - Units are SI (m, kg, s, N).  z is the vertical axis.
 */
#ifndef TITAN_H
#define TITAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct titan_sim titan_sim;     /* opaque, library-owned */

typedef enum {
    TITAN_OK = 0,
    TITAN_E_INVALID = 1,      /* an argument failed validation; nothing changed     */
    TITAN_E_CUDA = 2,         /* a CUDA call failed (maybe earlier asynchronous work) */
    TITAN_E_OOM = 3,          /* a device or pinned-host allocation failed          */
    TITAN_E_TIMEOUT = 4,      /* a bounded device-side wait gave up                 */
    TITAN_E_BUSY = 5,         /* another call on this handle is in progress         */
    TITAN_E_UNSUPPORTED = 6   /* valid request this build or device cannot serve    */
} titan_status;

/* Masses (Sec. III-B: one integrator thread per mass).
 * pos [n][3], vel [n][3] (NULL: at rest), mass [n] (> 0, finite),
 * fixed [n] (NULL: none; nonzero: the mass never moves, Sec. III-A). */
typedef struct {
    uint32_t n;
    const double *pos;
    const double *vel;
    const double *mass;
    const uint8_t *fixed;
} titan_masses;

/* Springs (Sec. III-B, Eq. 1).  ends [n][2] mass indices i != j (< masses.n);
 * k [n] stiffness >= 0; rest [n] rest length >= 0 (NULL: the initial
 * distance between the two masses); damping [n] axial dashpot >= 0 (NULL:
 * titan_params.damping for every spring).  A rest length of 0 is legal on
 * every kernel: the spring pulls its ends together with force k l, and while
 * they coincide (l = 0) it has no axis and exerts no force. */
typedef struct {
    uint32_t n;
    const uint32_t *ends;
    const double *k;
    const double *rest;
    const double *damping;
} titan_springs;

typedef enum {
    TITAN_ACCUM_CSR = 0,      /* deterministic per-mass gather (fused, bit-exact)   */
    TITAN_ACCUM_ATOMIC = 1    /* per-spring scatter with vector atomics (Sec. III-B) */
} titan_accumulate;

typedef enum {
    TITAN_ORDER_INPUT = 0,    /* keep the caller's mass order on the device         */
    TITAN_ORDER_MORTON = 1    /* spatial order: 4x4x2 grid tiles when the masses sit on a
                                 grid (pitch = shortest spring), else a Morton curve */
} titan_order;

typedef enum {
    TITAN_EXEC_AUTO = 0,      /* persistent kernel when the system fits one cluster's
                                 shared memory and each CTA's rows are short (small
                                 systems), else launches; CSR accumulation only  */
    TITAN_EXEC_LAUNCH = 1,    /* one fused kernel launch per step (graph-captured)  */
    TITAN_EXEC_PERSISTENT = 2 /* one launch runs many steps (cluster, shared memory);
                                 titan_create returns TITAN_E_UNSUPPORTED if the
                                 system does not fit                               */
} titan_exec;

/* Integration parameters.  Fill with titan_default_params() first. */
typedef struct {
    double dt;                /* time step (s), > 0                                */
    double gravity[3];        /* m/s^2; default (0, 0, -9.81)                      */
    int32_t ground;           /* nonzero: ground plane z = 0 with friction         */
    double ground_k;          /* penalty stiffness (N/m), >= 0; default 1e5        */
    double mu;                /* Coulomb friction coefficient, >= 0; default 0.5   */
    double damping;           /* dashpot used when springs.damping is NULL         */
    int32_t accumulate;       /* titan_accumulate; default CSR                     */
    int32_t order;            /* titan_order; default MORTON                       */
    int32_t exec;             /* titan_exec; default AUTO                          */
    int32_t device;           /* CUDA device ordinal; default 0                    */
    void *stream;             /* cudaStream_t for the step loop; NULL: own stream  */
    uint64_t spin_limit;      /* bound on device spin-wait iterations; 0: default  */
    int32_t graph_chunk;      /* steps per captured CUDA graph; 0: 64; < 0: none   */
    int32_t kernel_variant;   /* CSR kernel: 0 auto (6 for masses on a grid when
                                 it fits, else 4 when it fits, else 3),
                                 1 direct loads, 2 TMA-staged stream, 3 bulk L2
                                 prefetch, 4 halo tables in shared memory, 5 halo +
                                 TMA-staged stream, 6 grid-box tables (masses on a
                                 cubic grid, at most one per cell; no neighbour
                                 index in the stream), 7 grid box + TMA-staged
                                 stream, 8 cube (springs inside a 256-mass cube
                                 read and evaluated once; 26-neighbour springs on
                                 a grid, at most one per mass and offset), 9 grid
                                 box with each warp's stream fed through a ring
                                 of bulk copies in shared memory, 10 two-phase
                                 cube (as 8: every spring in a cube evaluated
                                 once, forces exchanged through shared memory
                                 in direction groups).  4 to 10 return
                                 TITAN_E_UNSUPPORTED if their tables do not fit
                                 or their layout conditions fail            */
    int32_t l2_persist;       /* nonzero (default): keep the two state buffers of a
                                 CSR simulation resident in L2 (an access-policy
                                 window on the grid-box, cube and halo step
                                 kernels, taken only when both buffers fit the
                                 persisting part of L2; the context's
                                 persisting-L2 limit is raised while any such
                                 handle lives and restored by titan_destroy)    */
    int32_t launch_overlap;   /* nonzero (default): the grid-box and halo step
                                 kernels are launched as programmatic dependents
                                 of the previous step, so a step's CTAs start
                                 (and fetch their stream) while the previous
                                 step's last CTAs finish; they read the state
                                 only once it is complete.  0: plain stream
                                 order.  No result depends on it (bit for bit) */
    int32_t reserved[4];      /* zero                                              */
} titan_params;

/* Writes the defaults listed above into *p (p != NULL). */
void titan_default_params(titan_params *p);

/* Builds a simulation on the GPU (Sec. III-C: all objects live on the GPU).
 * Validates every input (indices in range, i != j, finite values, mass > 0,
 * dt > 0, k/rest/damping >= 0) before touching the device, copies the inputs
 * to device memory in the chosen layout, and sets *out.  The state is at
 * step 0 (t = 0).  Errors: TITAN_E_INVALID (bad input, *out untouched),
 * TITAN_E_OOM, TITAN_E_CUDA. */
titan_status titan_create(const titan_masses *masses, const titan_springs *springs,
                          const titan_params *params, titan_sim **out);

/* Enqueues n_steps time steps on the simulation's stream and returns without
 * waiting for them (Sec. III-D: the GPU runs while the caller continues).
 * Each step is the spring pass and the mass pass of Sec. III-B.  Steps are
 * replayed from captured CUDA graphs (params.graph_chunk): a count that is
 * not one graph of the ladder 64, 32, ..., 2 and is at most twice the chunk
 * gets a graph of its own, captured on its first use (the four most
 * recently used counts are kept), so a caller stepping by a fixed count
 * pays the capture once.  n_steps == 0 is a no-op.  Errors: TITAN_E_CUDA, TITAN_E_TIMEOUT (a bounded
 * device wait in the persistent kernel expired; reported by this or a later
 * call once the GPU has run it). */
titan_status titan_step(titan_sim *sim, uint64_t n_steps);

/* Takes a snapshot of the state after all steps enqueued so far, without
 * stalling the step loop: a device-side copy on the simulation stream, then a
 * device-to-host copy on `stream` (a cudaStream_t; NULL: a library-owned side
 * stream) into one of two pinned host buffers.  *ticket identifies it.
 * Only the two most recent snapshots are retained.  Errors: TITAN_E_CUDA. */
titan_status titan_snapshot_async(titan_sim *sim, void *stream, uint64_t *ticket);

/* Waits for snapshot `ticket` and returns pointers to library-owned arrays in
 * the caller's mass order: *pos and *vel are [n][3] float, *t the simulated
 * time of the snapshot (any output pointer may be NULL).  The arrays stay valid
 * until the second next titan_snapshot_async call or titan_destroy.
 * Errors: TITAN_E_INVALID (ticket unknown or already overwritten),
 * TITAN_E_CUDA. */
titan_status titan_snapshot_wait(titan_sim *sim, uint64_t ticket, const float **pos,
                                 const float **vel, double *t);

/* Sets sinusoidal actuation on the listed springs (Sec. V-B: springs expand
 * and contract over time; Sec. III-F edits pushed between steps):
 * rest(t) = L0 (1 + amp sin(2 pi freq_hz t + phase)), t = step * dt at the start
 * of the step.  amp == 0 turns actuation off for that spring.  freq_hz applies
 * to the whole system.  Takes effect from the next enqueued step.
 * Errors: TITAN_E_INVALID (index out of range, non-finite value). */
titan_status titan_set_actuation(titan_sim *sim, uint32_t n, const uint32_t *spring_ids,
                                 const float *amp, const float *phase, float freq_hz);

/* titan_set_actuation for every spring at once from DEVICE arrays (the
 * simulation's device): amp_dev[s] and phase_dev[s] for spring s in caller
 * order, n floats each; n must equal the simulation's spring count (n_springs
 * at creation plus springs added since).  The call checks every value on
 * the device, then copies the arrays into the library (it waits for both on
 * the simulation's stream, so the caller may reuse or free the arrays once
 * it returns; work the caller enqueued on other streams that writes them
 * must be complete).  Nothing changes on error.  Takes effect from the next
 * enqueued step.  The paper has no counterpart:
 * it keeps an optimisation loop's actuation on the GPU between rollouts.
 * Errors: TITAN_E_INVALID (n not the spring count, null array with n > 0,
 * non-finite value or freq_hz), TITAN_E_CUDA. */
titan_status titan_set_actuation_dev(titan_sim *sim, uint32_t n, const float *amp_dev, const float *phase_dev,
                                     float freq_hz);

/* Worm actuation (Sec. V-B, Eqs. 3-5): rest(t) = L0 (1 + c[s] sin(omega tau)),
 * tau = (t - t_offset[s]) mod period (floor modulo, in [0, period)).  c == 0
 * turns a spring off.  Replaces any sinusoidal actuation.  Takes effect from
 * the next enqueued step.  Errors: TITAN_E_INVALID. */
titan_status titan_set_worm_actuation(titan_sim *sim, uint32_t n, const uint32_t *spring_ids,
                                      const float *c, const float *t_offset, float omega, float period);

/* ---- edits between steps (Sec. III-C: O(1) insertion and deletion; Sec.
 * III-F: spring constants, rest lengths and topology changed while the
 * simulation runs).  Ids are the caller's: springs and masses added later get
 * the next free ids.  Parameter edits and removals patch the device arrays in
 * place (O(1) per spring).  Additions are queued and the device layout is
 * rebuilt, keeping the state, the step counter and the actuation, before the
 * next call that uses the state (O(masses + springs) once per batch of
 * additions); that rebuild invalidates earlier snapshot tickets. */

/* New stiffness, rest length and/or dashpot (any array may be NULL = keep). */
titan_status titan_set_spring_params(titan_sim *sim, uint32_t n, const uint32_t *spring_ids,
                                     const double *k, const double *rest, const double *damping);

/* Removes springs: their stiffness, dashpot and actuation become 0 (the paper's
 * lazy deletion); the ids stay reserved. */
titan_status titan_remove_springs(titan_sim *sim, uint32_t n, const uint32_t *spring_ids);

/* Adds springs (ends [n][2] ids of existing or added masses); rest NULL: the
 * distance between the two masses when the layout is rebuilt; damping NULL:
 * params.damping.  *first_id (may be NULL) receives the first new id. */
titan_status titan_add_springs(titan_sim *sim, uint32_t n, const uint32_t *ends, const double *k,
                               const double *rest, const double *damping, uint32_t *first_id);

/* Adds masses (pos [n][3], vel [n][3] or NULL, mass [n], fixed [n] or NULL). */
titan_status titan_add_masses(titan_sim *sim, uint32_t n, const double *pos, const double *vel,
                              const double *mass, const uint8_t *fixed, uint32_t *first_id);

/* Fixes (nonzero) or frees masses (Sec. III-A constraints). */
titan_status titan_set_fixed(titan_sim *sim, uint32_t n, const uint32_t *mass_ids, const uint8_t *fixed);

/* Replaces the positions and velocities (host FP64 arrays [n][3], caller
 * order; vel NULL: zero) from the next enqueued step on; the step counter is
 * kept.  Used to resume from a checkpoint (Sec. III-D breakpoints).
 * Errors: TITAN_E_INVALID (non-finite), TITAN_E_CUDA. */
titan_status titan_set_state(titan_sim *sim, const double *pos, const double *vel);

/* Writes the state after all steps enqueued so far, in the caller's mass
 * order, into caller-provided DEVICE arrays pos_dev and vel_dev ([n][3]
 * float; either may be NULL), ordered on the simulation stream; when `stream`
 * (a cudaStream_t) is non-NULL it is made to wait for the copy.  Does not block
 * the host.  Errors: TITAN_E_CUDA. */
titan_status titan_read_state_dev(titan_sim *sim, float *pos_dev, float *vel_dev, void *stream);

/* Group centroids of the state after all steps enqueued so far (the objective
 * of a swarm of robots simulated as one system, Sec. V-B: how far each moved).
 * Group g is the masses with caller indices first_dev[g] .. first_dev[g+1] - 1
 * (first_dev: DEVICE uint32 array of n_groups + 1 non-decreasing offsets, the
 * last at most n_masses).  out_dev[g][0..2] (DEVICE float) = the mean
 * position of the group, summed in FP64 mass by mass, minus origin_dev[g][..]
 * when origin_dev (DEVICE float [n_groups][3]) is non-NULL; an empty group
 * gives 0.  Enqueued on the simulation stream.  Offsets are not read on the
 * host: out-of-range ones are clamped to n_masses.  Errors: TITAN_E_INVALID
 * (null array with n_groups > 0), TITAN_E_CUDA. */
titan_status titan_group_centroids(titan_sim *sim, uint32_t n_groups, const uint32_t *first_dev,
                                   const float *origin_dev, float *out_dev);

/* The adjoint seed of sum_g w[g] * (centroid of group g) . e_axis:
 * seed_dev[i][axis] = w_dev[g] / (number of masses of group g) for every mass
 * i of group g, every other entry of seed_dev ([n_masses][3], DEVICE float)
 * 0.  Groups as for titan_group_centroids; axis 0, 1 or 2.  Enqueued on the
 * simulation stream.  Errors: TITAN_E_INVALID, TITAN_E_CUDA. */
titan_status titan_group_seed(titan_sim *sim, uint32_t n_groups, const uint32_t *first_dev, const float *w_dev,
                              int32_t axis, float *seed_dev);

/* Sets the step counter (the simulated time is steps * dt; the actuation
 * clock reads it) for the steps enqueued from now on.  Errors: TITAN_E_CUDA. */
titan_status titan_set_step(titan_sim *sim, uint64_t step);

/* Reverse-mode derivative of a rollout (gradient-based design of actuated
 * robots; the paper's Sec. III-F shape and actuation optimisation done with
 * gradients).  From the current state and step, runs n_steps ordinary steps
 * (the simulation advances as titan_step would), keeping the state every
 * `every` steps (0: 50), then recomputes each segment from its checkpoint and
 * reverses it, accumulating
 *   grad_amp_dev[s]   = dJ / dA_s,    grad_phase_dev[s] = dJ / dphi_s
 * for J = sum_i seed_pos[i] . x_T[i] + seed_vel[i] . v_T[i] (x_T, v_T: the
 * state after the rollout).  All arrays are DEVICE float arrays in caller
 * order: seed_pos_dev and seed_vel_dev [n][3] (seed_vel_dev may be NULL),
 * gradients [n_springs] (overwritten).  Requires CSR accumulation and
 * actuation set with titan_set_actuation or titan_set_actuation_dev.  At the
 * kinks of contact and friction the derivative of the branch the forward step
 * took is used.
 * Enqueued on the simulation stream.  Errors: TITAN_E_INVALID,
 * TITAN_E_UNSUPPORTED (atomic accumulation), TITAN_E_OOM, TITAN_E_CUDA. */
titan_status titan_adjoint(titan_sim *sim, uint64_t n_steps, uint32_t every, const float *seed_pos_dev,
                           const float *seed_vel_dev, float *grad_amp_dev, float *grad_phase_dev);

/* Blocks until every enqueued step and copy has finished (the paper's
 * waitForEvent, Sec. III-D).  Errors: TITAN_E_CUDA, TITAN_E_TIMEOUT. */
titan_status titan_sync(titan_sim *sim);

/* Number of steps enqueued so far (the simulated time is steps * dt). */
uint64_t titan_steps(const titan_sim *sim);

/* How titan_step runs, as resolved from params.exec: TITAN_EXEC_PERSISTENT
 * (chunks of up to 65,536 steps per launch of one thread-block cluster that
 * holds the whole system in shared memory) or TITAN_EXEC_LAUNCH (one fused
 * kernel per step, graph-captured); -1 for a NULL handle.  Re-resolved when
 * actuation or per-spring damping enlarges the entries and after a layout
 * rebuild; an edit that no longer fits falls back to launches. */
int32_t titan_exec_mode(const titan_sim *sim);

/* The step kernel titan_create resolved params.kernel_variant to: 1..8 as
 * listed for kernel_variant (never 0), 0 for atomic accumulation, -1 for a
 * NULL handle.  The resolution is redone when added masses or springs force a
 * layout rebuild. */
int32_t titan_csr_kernel(const titan_sim *sim);

/* Text of the last error on this handle, or of the last failed titan_create
 * on this thread when sim is NULL.  Owned by the library; never NULL. */
const char *titan_last_error(const titan_sim *sim);

/* One time step of the atomic-scatter kernels on caller-owned device arrays,
 * for callers that cannot allocate device memory: a control loop with a hard
 * per-step deadline (cudaMalloc and cudaFree may synchronise the device and
 * take unbounded time), or a plug-in inside a host framework that owns all
 * device memory through its own pool.  The call allocates nothing; the
 * per-mass force accumulator it needs is a fixed 4 MiB array inside the
 * library (every GPU that loads the library holds it until the process exits).
 * The paper has no counterpart of this call.
 *
 * Inputs (device pointers, caller order, float): pos_dev and vel_dev [n][3],
 * inv_mass_dev [n] (0 marks a fixed mass), ends_dev [n_springs][2] (u32),
 * k_dev and rest_dev [n_springs]; damping is the dashpot of every spring.
 * params supplies dt, gravity, ground, ground_k and mu (other fields unused).
 * Outputs: pos_out_dev and vel_out_dev [n][3] (must not alias the inputs).
 * Enqueued on `stream` (a cudaStream_t; NULL: the legacy default stream) on
 * the current device; the call does not wait for it.
 * Limits: n_masses <= 262144; larger counts return TITAN_E_INVALID.
 * The first call on each device (and the first after the device's context is
 * recreated, e.g. by cudaDeviceReset) looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  All calls share the one array per device and each call
 * clears the part it uses first: calls whose work overlaps on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * Spring ends must be < n_masses and distinct.  They are device data, so the
 * kernel checks them: a spring that breaks this is skipped (nothing is read or
 * written through it) and counted; the next call first waits for the work
 * queued on its stream, reads and clears that count and, if it is nonzero,
 * returns TITAN_E_INVALID without stepping.
 * Errors: TITAN_E_INVALID (sizes, null pointers, dt/damping, bad spring ends
 * in the previous call), TITAN_E_CUDA; the text is in titan_last_error(NULL). */
titan_status titan_step_atomic_noalloc(uint32_t n_masses, const float *pos_dev, const float *vel_dev,
                                       const float *inv_mass_dev, uint32_t n_springs,
                                       const uint32_t *ends_dev, const float *k_dev,
                                       const float *rest_dev, float damping,
                                       const titan_params *params, float *pos_out_dev,
                                       float *vel_out_dev, void *stream);

/* Failure-path self-test of the bounded device waits (no counterpart in the
 * paper; it backs the TITAN_E_TIMEOUT contract above).  Launches one CTA on
 * `device` whose thread waits on an mbarrier that nothing arrives on, polling
 * at most spin_limit times (1 <= spin_limit <= 2^20), and synchronises.
 * Returns TITAN_E_TIMEOUT when the wait expired and the device flag reached
 * the host - the expected outcome, after which the device stays usable;
 * TITAN_E_INVALID for an out-of-range spin_limit; TITAN_E_CUDA otherwise.
 * Allocates and frees one int of device memory; uses the legacy stream. */
titan_status titan_selftest_wait_timeout(int32_t device, uint32_t spin_limit);

/* Waits for outstanding work and frees every resource of the handle.
 * NULL is a no-op.  Returns the status of that final wait. */
titan_status titan_destroy(titan_sim *sim);

/* ------------------------------------------------------------------ batches
 * Many independent systems (robots) advanced together: the paper's parallel
 * robots and agents (Sec. I; Sec. V-B, 100 worms simulated at once).  Each
 * system is owned by one thread-block cluster whose shared memory holds its
 * state and springs for a whole rollout; the clusters of one size and
 * shared-memory class run in one persistent launch (small systems share an
 * SM), and the launches of a rollout form one CUDA graph.
 * Systems keep their own mass order; masses of different systems never
 * interact. */
typedef struct titan_batch titan_batch;

/* Sinusoidal actuation of one system's springs (Sec. V-B):
 * rest(t) = L0 (1 + amp[s] sin(2 pi freq_hz t + phase[s])); amp NULL: none. */
typedef struct {
    const double *amp;
    const double *phase;
    double freq_hz;
} titan_actuation;

/* Builds a batch of n_systems systems (masses[r], springs[r], act[r]; act
 * may be NULL).  params supplies dt, gravity, ground, ground_k, mu, damping
 * (uniform: per-spring damping returns TITAN_E_UNSUPPORTED), device, stream
 * and spin_limit.  Every system must fit a cluster of 8 CTAs (about 30,000
 * springs); all actuated systems share one frequency.  Errors:
 * TITAN_E_INVALID, TITAN_E_UNSUPPORTED, TITAN_E_OOM, TITAN_E_CUDA. */
titan_status titan_batch_create(uint32_t n_systems, const titan_masses *masses,
                                const titan_springs *springs, const titan_actuation *act,
                                const titan_params *params, titan_batch **out);

/* Enqueues a rollout of n_steps (< 2^32) steps of every system and returns
 * without waiting.  The actuation clock continues across rollouts. */
titan_status titan_batch_rollout(titan_batch *b, uint64_t n_steps);

/* The autotuner: times each launch group with 128, 256, 512 and 1024 threads
 * per CTA and at most 1, 2, 4 or 8 threads per mass over a probe_steps
 * rollout (0: 50) and keeps the fastest pair.  The state is unchanged. */
titan_status titan_batch_autotune(titan_batch *b, uint32_t probe_steps);

/* Sets a launch group's shape by hand: threads per CTA (a multiple of 32,
 * up to 1024) and the most threads per mass (1, 2, 4 or 8): a mass's springs
 * are split over that many threads, and each CTA takes the largest power of
 * two up to it that still gives every mass of the CTA its own threads in one
 * pass (at least 1).  Errors: TITAN_E_INVALID. */
titan_status titan_batch_configure(titan_batch *b, uint32_t group, uint32_t threads,
                                   uint32_t threads_per_mass);

/* Restores every system's initial state and the step counter to 0. */
titan_status titan_batch_reset(titan_batch *b);

/* Waits for the batch's work; TITAN_E_TIMEOUT if a bounded wait expired. */
titan_status titan_batch_sync(titan_batch *b);

/* Copies system `system`'s current positions and velocities ([n][3] float,
 * its own mass order; either may be NULL) to host memory.  Waits. */
titan_status titan_batch_read(titan_batch *b, uint32_t system, float *pos, float *vel);

/* Writes every system's centroid ([n_systems][3] float, host) after the
 * enqueued work.  Waits. */
titan_status titan_batch_centroids(titan_batch *b, float *out);

/* Number of launch groups (one per cluster size) and, per group, its cluster
 * size, threads per CTA, most threads per mass and CTA count (outputs may be
 * NULL). */
uint32_t titan_batch_groups(const titan_batch *b);
titan_status titan_batch_info(const titan_batch *b, uint32_t group, uint32_t *cluster,
                              uint32_t *threads, uint32_t *threads_per_mass, uint32_t *ctas);

/* The launch group (0 .. titan_batch_groups - 1) whose launches advance
 * system `system`.  TITAN_E_INVALID for a null batch or output, or a system
 * index out of range. */
titan_status titan_batch_system_group(const titan_batch *b, uint32_t system, uint32_t *group);

/* Text of the last error on this batch ("" if none). */
const char *titan_batch_last_error(const titan_batch *b);

/* Waits and frees the batch.  NULL is a no-op. */
titan_status titan_batch_destroy(titan_batch *b);

/* ------------------------------------------------------------------ surrogate
 * A fitness-surrogate MLP (in -> hidden -> hidden -> hidden -> 1, GELU after
 * each hidden layer) trained and evaluated on the tcgen05 tensor cores with
 * BF16 operands and FP32 accumulation.  It pre-screens candidate robots in a
 * morphology search whose survivors the simulator scores (the paper's
 * Sec. III-F shape and topology optimisation, with a learned filter).
 * Parameters are FP32 (layout: W1^T [hidden][in], b1, W2^T [hidden][hidden],
 * b2, W3^T, b3, w4 [hidden], b4); activations BF16.  Batches are multiples
 * of 128; in and hidden are multiples of 128.  Device pointers throughout. */
typedef struct titan_mlp titan_mlp;

/* C[M][N] = A[M][K] B[N][K]^T on the tensor cores: A and B row-major BF16
 * (uint16 bit patterns, 16-byte aligned), C row-major FP32, all on the
 * current device.  M and N multiples of 128, K of 64.  Enqueued on `stream`
 * (NULL: the legacy default stream); returns without waiting.  A kernel
 * whose bounded wait expires sets a per-device flag in pinned host memory;
 * the next titan_gemm_bf16_tn or titan_gemm_check on that device reads it
 * without waiting, clears it and returns TITAN_E_TIMEOUT (that call enqueues
 * nothing).  Errors: TITAN_E_INVALID, TITAN_E_CUDA, TITAN_E_TIMEOUT. */
titan_status titan_gemm_bf16_tn(uint32_t M, uint32_t N, uint32_t K, const uint16_t *A_dev,
                                const uint16_t *B_dev, float *C_dev, void *stream);

/* Reads (and clears) the current device's GEMM flag: TITAN_E_TIMEOUT if a
 * titan_gemm_bf16_tn kernel gave up on a bounded wait.  Call it after
 * synchronising the streams the GEMMs ran on to see every such failure. */
titan_status titan_gemm_check(void);

titan_status titan_mlp_create(uint32_t in, uint32_t hidden, uint64_t seed, int32_t device, void *stream,
                              titan_mlp **out);
uint64_t titan_mlp_param_count(const titan_mlp *m);
titan_status titan_mlp_get_params(titan_mlp *m, float *host_params);
titan_status titan_mlp_set_params(titan_mlp *m, const float *host_params);

/* y_dev[b] = network(x_dev[b][:]) for a batch of BF16 inputs. */
titan_status titan_mlp_forward(titan_mlp *m, const uint16_t *x_dev, uint32_t batch, float *y_dev);

/* Mean-squared-error loss against t_dev and its gradient with respect to
 * every parameter (flat FP32, the parameter layout; grad_dev may be NULL). */
titan_status titan_mlp_gradient(titan_mlp *m, const uint16_t *x_dev, const float *t_dev, uint32_t batch,
                                float *loss_dev, float *grad_dev);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the batch's gradient;
 * loss_dev (may be NULL) receives the batch loss.  Enqueued, not waited for. */
titan_status titan_mlp_train_step(titan_mlp *m, const uint16_t *x_dev, const float *t_dev, uint32_t batch,
                                  float lr, float *loss_dev);
titan_status titan_mlp_sync(titan_mlp *m);
const char *titan_mlp_last_error(const titan_mlp *m);
titan_status titan_mlp_destroy(titan_mlp *m);

#ifdef __cplusplus
}
#endif
#endif /* TITAN_H */
