/*
 * ilg.h — C ABI of libilg.so, the GB300 (sm_103a) implementation of the
 * over-relaxed diffusive integer lattice gas of Strand & Wagner,
 * "Over-Relaxation in Diffusive Integer Lattice Gas" (arXiv 2203.01380).
 *
 * One time step, for every node x of a periodic D1Q3, D2Q5 or D2Q9 lattice:
 *   flip      m_i = n_{-i}(x,t) when omega_eff > 1            (Sec. III, Eq. flip)
 *   collide   sampling collision with fraction omega*:         (Sec. II; Sec. III, Eq. LGflip)
 *             binomial thinning, multinomial redistribution
 *             with weights w_i; mass conserved exactly         (Sec. II, Eq. 2)
 *             (D2Q9, the paper's D1Q3 extended to the product
 *             lattice: see theta below)
 *   stream    n_i(x + v_i, t+1) = n'_i(x)                      (Sec. II, Eq. ilgeq)
 * with omega^j = 2 - omega* above omega_eff = 1                 (Sec. IV, Eq. omegaj).
 *
 * Conventions
 *   - Occupations are uint16, stored as Q planes n[i][y][x] (x fastest), velocity
 *     order rest first: D1Q3 (0, +1, -1); D2Q5 (0, +x, -x, +y, -y), y = row;
 *     D2Q9 (0, +x, -x, +y, -y, (+1,+1), (-1,-1), (+1,-1), (-1,+1)).
 *   - The library owns the device memory of a context; the caller owns every host
 *     array it passes and keeps it alive for the duration of the call.
 *   - Calls on one context are not thread-safe; different contexts are independent.
 *   - Every call returns an ilg_status; no C++ exception crosses the ABI.
 *     ilg_last_error() describes the last failure on a context.
 *   - "stream" is a cudaStream_t (NULL = the legacy default stream).  Kernels of a
 *     context run on its stream; calls that return host data synchronise it.
 *   - Random numbers: Philox4x32-10, key = seed, counter = (step t, node x + Lx*y,
 *     replica, purpose tag and block).  Results do not depend on launch shape,
 *     stream, batching or placement.
 */
#ifndef ILG_H
#define ILG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ILG_OK = 0,
  ILG_E_INVALID = 1,  /* bad argument or parameter */
  ILG_E_OOM = 2,      /* device allocation failed */
  ILG_E_OVERFLOW = 3, /* some occupation would exceed 65535; state rolled back */
  ILG_E_CUDA = 4,     /* CUDA runtime error */
  ILG_E_TIMEOUT = 5,  /* a bounded device wait gave up */
  ILG_E_STATE = 6     /* call out of order (e.g. step before init/set_state) */
} ilg_status;

typedef enum { ILG_D1Q3 = 1, ILG_D2Q5 = 2, ILG_D2Q9 = 3 } ilg_lattice;

/* Parameters of one lattice (Sec. II-V).
 *   lattice        ILG_D1Q3, ILG_D2Q5 or ILG_D2Q9 (D2Q9: contexts and the comparator;
 *                  batches take D1Q3 rings, the server D2Q5 lattices, temporal blocking D2Q5)
 *   Lx, Ly         periodic extent, >= 3 each (Ly is ignored and taken as 1 for D1Q3);
 *                  Lx * Ly < 2^32
 *   n0, amp        initial state (Sec. V): see init_weighted
 *   mode_mx/my     wave numbers of the initial sine, k = 2 pi (mx/Lx, my/Ly); at most
 *                  one of them nonzero (an axis mode)
 *   init_weighted  1: mean of velocity i is w_i (Q n0 + amp sin(k.x))  (Sec. V, w_i P(rho));
 *                  0: mean of every velocity is n0 + amp sin(k.x) / Q
 *                  every mean must lie in [0, 700]
 *   omega_eff      in (0, 2]: <= 1 collision fraction omega* = omega_eff without flip;
 *                  > 1 flip on and omega* = 2 - omega_eff, so omega^j = omega_eff
 *   theta          D1Q3 weights (1-theta, theta/2, theta/2), theta in (0, 1);
 *                  D2Q5 weights (1-2 theta, theta/2 x4), theta in (0, 1/2];
 *                  D2Q9 weights the products of the D1Q3 ones in x and y: (1-theta)^2,
 *                  theta (1-theta)/2 x4 (axis), theta^2/4 x4 (diagonal), theta in (0, 1);
 *                  its moving particles split binomially into axis and diagonal ones
 *                  with P = 4 w_axis / (1 - w_0) before their directions are drawn
 *   seed, replica  Philox key and the replica word of every counter
 *   sampler        how the collision draws its random decisions (same law, different bits):
 *                  ILG_SAMPLER_BINOMIAL (0): per velocity one binomial draw of the
 *                    particles removed, one of those sent to rest, and one bit per
 *                    moving particle for its direction; each draw is one 32-bit word
 *                    through an integer alias table (the fast sampler)
 *                  ILG_SAMPLER_PARTICLE (1): every particle decides on its own
 *                    32-bit word against integer boundaries (stay, rest, each moving
 *                    velocity): the plain reference form, one word per particle */
typedef struct {
  int32_t lattice;
  uint32_t Lx;
  uint32_t Ly;
  int32_t mode_mx;
  int32_t mode_my;
  int32_t init_weighted;
  double n0;
  double amp;
  double omega_eff;
  double theta;
  uint64_t seed;
  uint32_t replica;
  uint32_t sampler;  /* ILG_SAMPLER_BINOMIAL or ILG_SAMPLER_PARTICLE */
} ilg_params;

enum { ILG_SAMPLER_BINOMIAL = 0, ILG_SAMPLER_PARTICLE = 1 };

typedef struct ilg_ctx ilg_ctx;

/* Create a context for one lattice: validates params, allocates two state buffers
 * (2 * Q * Lx * Ly uint16) plus tables and reduction scratch on the current device,
 * and builds the integer alias tables of the collision.  *out is NULL on failure. */
ilg_status ilg_create(const ilg_params* params, void* stream, ilg_ctx** out);

/* Release every device allocation of the context (after synchronising its stream). */
ilg_status ilg_destroy(ilg_ctx* ctx);

/* Message describing the last failure on ctx (empty string if none); valid until
 * the next call on ctx.  ilg_last_error(NULL) describes the last failed ilg_create. */
const char* ilg_last_error(const ilg_ctx* ctx);

/* Poisson initial state of Sec. V (means as in ilg_params), step counter t := 0.
 * ILG_E_INVALID if a mean lies outside [0, 700]. */
ilg_status ilg_init(ilg_ctx* ctx);

/* Copy a state in: host (pageable or pinned) or device array of n = Q*Lx*Ly uint16 in
 * the plane layout above, at step t (t < 2^32).  Synchronous. */
ilg_status ilg_set_state(ilg_ctx* ctx, const uint16_t* host, size_t n, uint64_t t);
ilg_status ilg_set_state_device(ilg_ctx* ctx, const uint16_t* dev, size_t n, uint64_t t);

/* Copy the current state out (n = Q*Lx*Ly) and its step counter (t may be NULL).
 * Synchronous. */
ilg_status ilg_get_state(ilg_ctx* ctx, uint16_t* host, size_t n, uint64_t* t);
ilg_status ilg_get_state_device(ilg_ctx* ctx, uint16_t* dev, size_t n, uint64_t* t);

/* Advance T time steps (t -> t + T; t + T must stay below 2^32).  Kernels are queued
 * on the context stream; the call then reads one overflow word back (synchronising
 * the stream).  On ILG_E_OVERFLOW the context holds the state and step counter of
 * the last completed step before the failing one. */
ilg_status ilg_step(ilg_ctx* ctx, uint32_t T);

/* Temporal blocking (D2Q5): with depth >= 2, ilg_step runs blocks of `depth` steps
 * per launch (square tiles of 44 - 2 depth nodes with a halo of depth nodes,
 * recomputed, held in shared memory) and single steps for the remainder; results
 * are bit-identical to single
 * steps.  depth 0 or 1 switches it off (the default); at most 8.  On
 * ILG_E_OVERFLOW the state is the input of the failing launch. */
ilg_status ilg_set_temporal_blocking(ilg_ctx* ctx, uint32_t depth);

/* Autotuner.  Times the launch shapes that give the same bits on a copy of the
 * current state (2 extra state buffers, freed before return) and keeps the fastest
 * for later ilg_step calls:
 *   candidate 0  row-tiled step, 8 nodes per thread (16-byte vectors), 3 blocks per SM
 *   candidate 1  row-tiled step, 4 nodes per thread (8-byte vectors), 3 blocks per SM
 *   candidate 2  node-parallel step, one node per thread
 *   candidate 3, 4  temporal blocking of depth 2, 4 (D2Q5; the remainder of a call
 *                takes the fastest single-step candidate)
 *   candidate 5  8-node vectors in warp segments: each warp walks 8192 nodes of a row,
 *                neighbours exchanged by shuffles, no block barrier
 *   candidate 6  8-node vectors in warp segments (rows a multiple of 8; both collision
 *                probabilities strictly between 0 and 1): every warp an equal share
 *                of the lattice's vectors, the next tile's occupations copied into
 *                shared memory while the current one collides, the flip a
 *                compile-time plane order, the fast collision branch-free, the
 *                values crossing a segment's ends written by the warp that computes
 *                them (no node computed twice); one block of 384 threads per SM
 *                (the default where it applies)
 *   candidate 7  as 6 with 4-node vectors (rows a multiple of 4), 640 threads per SM
 *                (the default where 6 does not apply and 7 does)
 *   D2Q9 lattices: candidate 2 (node-parallel, two nodes of a row per thread where
 *                rows are even) and the staged warp step with 4-node vectors (rows a
 *                multiple of 4; all three probabilities strictly between 0 and 1),
 *                collided two nodes at a time in shared memory, in 512 threads per SM
 *                (candidate 6, the default where it applies) or 640 (candidate 7)
 * Candidates that do not apply (row length, lattice, occupations that need the
 * general collision, the particle sampler) are skipped (ms_per_step < 0).  A choice that stops applying after
 * ilg_set_state (e.g. occupations rise) falls back to the default.  trial_steps:
 * steps per candidate (0: 20; at most 1000).  The state, the step counter and all
 * results are unchanged.  ILG_E_OOM if the scratch does not fit.  Synchronous.
 * ilg_set_temporal_blocking later overrides the depth. */
typedef struct {
  uint32_t choice;         /* index of the chosen candidate */
  uint32_t tb_depth;       /* contexts: temporal blocking depth now in use (0: none) */
  uint32_t threads;        /* threads per block of the choice */
  uint32_t n;              /* candidates considered */
  double ms_per_step[8];   /* measured ms per time step per candidate; < 0: not applicable */
} ilg_tuning;

ilg_status ilg_autotune(ilg_ctx* ctx, uint32_t trial_steps, ilg_tuning* out);
/* Set the single-step kernel by hand: candidate 0, 1, 2, 5, 6 or 7 as above, -1 the default.
 * A candidate that does not apply to the current state falls back to the default;
 * results are the same bits either way. */
ilg_status ilg_set_step_kernel(ilg_ctx* ctx, int32_t candidate);

/* Observables of the current state (Sec. V).  modes: nmodes pairs (mx, my), each an
 * axis mode (one of the two zero, not both).  For a mode along x with
 * D(x) = Lx*C(x) - M, C(x) = sum_y N(x,y), r = (mx*x) mod Lx:
 *   re = sum_x cos(2 pi r / Lx) D(x) / Lx,  im = sum_x sin(2 pi r / Lx) D(x) / Lx,
 *   amp = im / (Lx*Ly/2)  (A^LG of Sec. V),  Sk = (re^2 + im^2) / (Lx*Ly);
 * modes along y use row sums R(y) and Ly.  Integer sums are exact (int64); the
 * projections are compensated double-precision dot products.  Every output pointer
 * is a host array (nmodes entries for re/im/amp/Sk, Lx for col_sums, Ly for
 * row_sums) and may be NULL.  Synchronous. */
ilg_status ilg_observables(ilg_ctx* ctx, const int32_t* modes, uint32_t nmodes, uint64_t* t,
                           uint64_t* mass, double* re, double* im, double* amp, double* Sk,
                           int64_t* col_sums, int64_t* row_sums);

/* ---------------------------------------------------------------------------
 * Batched D1Q3 replicas (independent rings of differing length, occupation and
 * omega_eff, as the ensembles of Sec. V).  One persistent kernel launch, captured
 * in a CUDA graph, advances every ring: blocks take rings longest first, hold a
 * ring and its alias tables in shared memory for all steps, and write it back.
 * Results equal, bit for bit, those of one context per ring (ilg_create ...), as
 * every random number is keyed by the ring's replica word.  All rings of a batch
 * share one seed; Lx <= 10240 each.  Host arrays only; calls synchronise.
 *   ilg_batch_create   params: n D1Q3 parameter sets (replica i = params[i]); tables
 *                      and device memory for all rings (stream NULL: a private one)
 *   ilg_batch_init     Poisson initial state of every ring (as ilg_init), t := 0
 *   ilg_batch_set_state / get_state   ring i, 3*Lx uint16 (planes rest, +1, -1)
 *   ilg_batch_run      T steps for every ring; if amp_record != NULL it receives
 *                      n*T doubles, A^LG of mode record_mode of ring i after step s
 *                      at [i*T + s] (as ilg_observables' amp).  ILG_E_OVERFLOW: some
 *                      ring stopped at the step that would exceed 65535 (its state
 *                      and t are those before that step); the others completed
 *   ilg_batch_observables   per ring: mass[i] and A^LG of one mode amp[i]
 *   ilg_batch_ensemble T steps for every ring (as ilg_batch_run) while the complex
 *                      amplitude a_r(t) = re + i im of axis mode `mode` of every
 *                      ring r is recorded at the start (t = 0) and after each step
 *                      (re, im as ilg_observables: sum_x cos|sin(2 pi (mode x mod L)
 *                      / L) (L N(x) - M) / L), then reduced over the rings on the
 *                      device, per t = 0..T (stats: 6 (T+1) doubles, row k at
 *                      [k (T+1) + t]):  k = 0, 1  ensemble means of re and im;
 *                      k = 2, 3  sample variances of re and im (divisor n - 1);
 *                      k = 4, 5  real and imaginary parts of the connected
 *                      correlation sum_r (a_r(t) - <a(t)>) conj(a_r(0) - <a(0)>) / (n - 1).
 *                      With Poisson starts these are the replica averages of Sec. V
 *                      (<A^LG(t)> = mean im / (L/2)) and the dynamic structure
 *                      factor S(k, t) = k=4 row / L.  record (may be NULL) receives
 *                      the per-ring values, [(r (T+1) + t) 2 + {0: re, 1: im}].
 *                      Needs n >= 2 rings of one length L and mode not a multiple of
 *                      L (ILG_E_INVALID otherwise).  Sums in a fixed order.
 * --------------------------------------------------------------------------- */
typedef struct ilg_batch ilg_batch;
ilg_status ilg_batch_create(const ilg_params* params, uint32_t n, void* stream, ilg_batch** out);
ilg_status ilg_batch_destroy(ilg_batch* b);
const char* ilg_batch_last_error(const ilg_batch* b);
ilg_status ilg_batch_init(ilg_batch* b);
ilg_status ilg_batch_set_state(ilg_batch* b, uint32_t i, const uint16_t* host, size_t n, uint64_t t);
ilg_status ilg_batch_get_state(ilg_batch* b, uint32_t i, uint16_t* host, size_t n, uint64_t* t);
ilg_status ilg_batch_run(ilg_batch* b, uint32_t T, int32_t record_mode, double* amp_record);
/* As ilg_batch_run, and the state of every ring after every step (Sec. V's profile
 * followed in time) goes to state_record (host array of T * sum_i 3 L_i uint16, or
 * NULL): ring i's record starts at T * o_i, o_i = sum_{r < i} 3 L_r, and holds its
 * state after step s (planes rest, +1, -1 as ilg_batch_get_state) at T * o_i + 3 L_i s.
 * A ring that stopped on overflow has no record after the step it stopped before.
 * The device copy of the record is allocated by the call (ILG_E_OOM if it does not
 * fit) and kept for later calls. */
ilg_status ilg_batch_run_record(ilg_batch* b, uint32_t T, int32_t record_mode, double* amp_record,
                                uint16_t* state_record);
ilg_status ilg_batch_observables(ilg_batch* b, int32_t mode, uint64_t* mass, double* amp);
ilg_status ilg_batch_ensemble(ilg_batch* b, uint32_t T, int32_t mode, double* stats, double* record);
/* Batch autotuner: times the block shapes 256, 512 and 1024 threads (candidates 0-2;
 * ceil(L / threads) nodes of a ring per thread and step, as many blocks per SM as
 * shared memory allows) for trial_steps steps (0: 50; at most 10000) on copies of all
 * rings, and keeps the fastest for later runs.  States, step counters and results are
 * unchanged.  out may be NULL.  Synchronous. */
ilg_status ilg_batch_autotune(ilg_batch* b, uint32_t trial_steps, ilg_tuning* out);

/* ---------------------------------------------------------------------------
 * Serving loop for D2Q5 lattice requests (continuous batching).  A worker thread
 * admits requests in arrival order while a free slot and room in a device arena
 * of hbm_bytes (allocated once, here) allow, keeps admitted lattices resident, and
 * advances all of them together: one launch per time step, `quantum` steps per
 * round (fewer when a request needs fewer), so newcomers join the next round.  A
 * finished request's observables go to the result queue and, if final_state was
 * given, its state (5*Lx*Ly uint16) is copied there; its memory returns to the
 * arena.  Results equal those of the request run alone (ilg_create ...), bit for
 * bit.  All requests share the server's seed.  Host waits only (no device spin).
 *   ilg_server_create    seed, arena bytes, slots, quantum, stream (NULL: private)
 *   ilg_server_submit    thread-safe, returns at once; final_state must stay valid
 *                        until the request's result has been polled
 *   ilg_server_poll      up to cap finished results (and their count in *n)
 *   ilg_server_wait_idle until every submitted request has finished (ILG_E_TIMEOUT)
 *   ilg_server_stats     worker busy time (s), node updates done, peak residents
 * Result fields: id, status (ILG_OK, ILG_E_OVERFLOW: stopped before the step that
 * would exceed 65535, ILG_E_INVALID: bad initial means), t (final step counter),
 * mass, amp = A^LG and Sk = S(k) of mode (1, 0), times in seconds on the server's
 * clock: submitted, admitted, done.
 * --------------------------------------------------------------------------- */
typedef struct {
  uint64_t id;
  int32_t status;
  uint32_t reserved;
  uint64_t t;
  uint64_t mass;
  double amp;
  double Sk;
  double t_submit;
  double t_admit;
  double t_done;
} ilg_result;
typedef struct ilg_server ilg_server;
/* Admission order: arrival order (the default), or least work (Lx*Ly*steps) first —
 * shorter requests then finish sooner; with an endless stream above capacity a large
 * request may wait indefinitely. */
enum { ILG_ADMIT_FIFO = 0, ILG_ADMIT_SMALLEST = 1 };
ilg_status ilg_server_set_policy(ilg_server* s, int32_t policy);
ilg_status ilg_server_create(uint64_t seed, uint64_t hbm_bytes, uint32_t max_slots, uint32_t quantum, void* stream,
                             ilg_server** out);
ilg_status ilg_server_submit(ilg_server* s, uint64_t id, const ilg_params* params, uint32_t steps,
                             uint16_t* final_state);
ilg_status ilg_server_poll(ilg_server* s, ilg_result* out, uint32_t cap, uint32_t* n);
ilg_status ilg_server_wait_idle(ilg_server* s, double timeout_s);
ilg_status ilg_server_stats(ilg_server* s, double* busy_s, double* node_updates, uint32_t* peak_resident);
ilg_status ilg_server_destroy(ilg_server* s);
const char* ilg_server_last_error(const ilg_server* s);

/* ---------------------------------------------------------------------------
 * Lattice Boltzmann comparator: the multi-relaxation-time lattice Boltzmann
 * equation that the lattice gas averages to (Sec. IV, Eq. MRTLB), in double
 * precision on the same lattices:
 *   f_i(x + v_i, t+1) = f_i^0 + sum_a w_i m_i^a (1 - omega^a) sum_j m_j^a (f_j - f_j^0),
 *   f_i^0 = w_i rho,  rho = sum_i f_i,
 * with m_i^a a transform matrix orthonormal under the weights (Sec. IV, Eq.
 * transform for D1Q3), omega^j for the current (odd) moments and omega for the
 * other non-conserved (even) moments.  The lattice gas with omega_eff > 1 has
 * omega^j = omega_eff, omega = 2 - omega_eff (Sec. IV, Eq. omegaj); with
 * omega_eff <= 1 both equal omega_eff.  Started from the means of the gas's
 * Poisson initial state it gives the gas's ensemble mean at every step.
 *
 * Parameters: lattice, Lx, Ly, mode_mx, mode_my, init_weighted, n0, amp, theta as
 * in ilg_params (they define the initial f = the Poisson means lambda_i(x), which
 * must lie in [0, 700]); omega_j and omega in [0, 2].
 * State: Q planes f[i][y][x] of doubles, same order as the gas.  The library owns
 * the device memory (two state buffers of Q*Lx*Ly doubles); the caller owns host
 * arrays.  Calls on one object are not thread-safe; every call returns a status,
 * ilg_lb_last_error describes the last failure (ilg_lb_last_error(NULL): the last
 * failed ilg_lb_create). */
typedef struct {
  int32_t lattice;
  uint32_t Lx;
  uint32_t Ly;
  int32_t mode_mx;
  int32_t mode_my;
  int32_t init_weighted;
  double n0;
  double amp;
  double omega_j;
  double omega;
  double theta;
} ilg_lb_params;

typedef struct ilg_lb ilg_lb;

ilg_status ilg_lb_create(const ilg_lb_params* params, void* stream, ilg_lb** out);
ilg_status ilg_lb_destroy(ilg_lb* lb);
const char* ilg_lb_last_error(const ilg_lb* lb);
/* The comparator's rates for the lattice gas with parameter omega_eff (Sec. IV, Eq.
 * omegaj): omega_eff > 1 (the flip on, collision fraction omega* = 2 - omega_eff)
 * gives omega_j = omega_eff for the current and omega = omega* for the other
 * non-conserved moments; omega_eff <= 1 gives omega_j = omega = omega_eff.  Host
 * only.  ILG_E_INVALID unless omega_eff lies in (0, 2] and both outputs are non-NULL. */
ilg_status ilg_lb_rates(double omega_eff, double* omega_j, double* omega);
/* f := lambda (the gas's Poisson means, Sec. V), t := 0. */
ilg_status ilg_lb_init(ilg_lb* lb);
/* Copy a state in or out (host arrays of n = Q*Lx*Ly doubles); synchronous. */
ilg_status ilg_lb_set_state(ilg_lb* lb, const double* host, size_t n, uint64_t t);
ilg_status ilg_lb_get_state(ilg_lb* lb, double* host, size_t n, uint64_t* t);
/* Advance T steps, queued on the object's stream (asynchronous). */
ilg_status ilg_lb_step(ilg_lb* lb, uint32_t T);
/* Mass M = sum f and, per axis mode (mx, my) (at most 256), with C the column
 * (row) sums of rho and r = (m x) mod L:
 *   re = sum_x cos(2 pi r / L) (C(x) - M / L),  im = sum_x sin(2 pi r / L) (C(x) - M / L),
 *   amp = im / (Lx*Ly/2)  (the measured amplitude of Sec. V).
 * Sums in a fixed order (deterministic), compensated.  Host outputs, each may be
 * NULL; synchronous. */
ilg_status ilg_lb_observables(ilg_lb* lb, const int32_t* modes, uint32_t nmodes, uint64_t* t, double* mass,
                              double* re, double* im, double* amp);

/* Observables of a state in caller-owned device memory, allocating nothing (the
 * paper has no counterpart; this serves callers that cannot allocate device memory
 * when they need the numbers: applications whose device memory all belongs to their
 * own pool, so that cudaMalloc would fail, and real-time loops that must not wait on
 * the allocator's locks or on the device-wide synchronisation of freeing memory).
 *   lattice, Lx, Ly  as in ilg_params (Ly taken as 1 for D1Q3); Lx, Ly <= 32768
 *   state            device array, Q*Lx*Ly uint16 in the plane layout above (read only)
 *   modes, nmodes    host array of nmodes <= 256 axis modes (mx, my), as ilg_observables
 *   stream           cudaStream_t the work runs on
 *   mass, re, im, amp, Sk   host outputs as in ilg_observables (each may be NULL)
 * The results equal those of ilg_observables on the same state.  Scratch lives in a
 * static device array of about 530 KB that every GPU which loads the library holds
 * until the process exits; nothing is allocated or freed.  The first call on a device
 * looks up that array's device address (with the device current) and caches it:
 * make that first call before any stream capture.  All calls share the one array and
 * each clears the sums it accumulates: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.  Sizes
 * beyond the limits give ILG_E_INVALID (message in ilg_last_error(NULL)).
 * Synchronous: returns after the results are on the host. */
ilg_status ilg_observables_noalloc(int32_t lattice, uint32_t Lx, uint32_t Ly, const uint16_t* state,
                                   const int32_t* modes, uint32_t nmodes, void* stream, uint64_t* mass,
                                   double* re, double* im, double* amp, double* Sk);

/* Diagnostics of the building blocks, for parity tests.
 * ilg_philox: n Philox4x32-10 blocks computed on the device; ctr (4n words) and out
 *   (4n words) are host arrays; key = (seed lo32, seed hi32).
 * ilg_binomial_table: the 2016-entry integer CDF table (rows n = 1..63, row n at
 *   offset n(n-1)/2) of Binomial(n, P / 2^32), 0 < P < 2^32; host only.
 * ilg_alias_table: the 4096-entry alias tables (rows n = 0..63 of 64 columns, column
 *   j of row n at offset 64 n + j) the collision draws Binomial(n, P / 2^32) with: a
 *   draw u takes column j = u >> 26 and yields j if u < thr[.], else alias[.]; they
 *   realise the CDF table's integer pmf exactly (outcomes above n get no draw).
 *   Host only.
 * ilg_poisson_table: the Poisson CDF table of the initial state for mean lambda;
 *   writes at most cap entries and their count to *K; host only. */
ilg_status ilg_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, size_t n, void* stream);
ilg_status ilg_binomial_table(uint64_t P, uint32_t* out);
ilg_status ilg_alias_table(uint64_t P, uint32_t* thr, uint32_t* alias);
ilg_status ilg_poisson_table(double lambda, uint32_t* out, uint32_t cap, uint32_t* K);

/* Integer throughput of the GPU, measured (the paper has no counterpart: these are
 * the denominators of the step kernels' integer roofline, whose random numbers and
 * table draws bound the step).  Kernels of fixed length on registers only, enough
 * warps on every SM to hide fixed latencies, eight independent chains per thread,
 * timed with CUDA events on `stream` over a region of `seconds` (0.05 .. 10) after a
 * calibration.  kind:
 *   0  Philox4x32-10 blocks per second (the generator of every step, with the
 *      step's counter layout: a launch-wide word, a per-thread word, constants)
 *   1  3-input logic (lop3) lane-operations per second
 *   2  32-bit multiply-add lane-operations per second
 *   3  32x32 -> 64-bit multiply-add lane-operations per second
 *   4  lane-operations per second of an even mix of kinds 1 and 2
 * *rate receives the figure, *ms (may be NULL) the timed region.  Synchronous.
 * ILG_E_INVALID for a bad kind or length (message in ilg_last_error(NULL)). */
ilg_status ilg_int_peak(int32_t kind, double seconds, void* stream, double* rate, double* ms);

/* Failure injection for tests of the error paths (the paper has no counterpart).
 * After `after` more successful device allocations made by the library (contexts,
 * batches, the server's arena and buffers, the comparator, scratch), the next one
 * reports failure without calling the allocator, so that call returns ILG_E_OOM
 * having released what it had allocated; then injection is off again.  after < 0
 * switches it off.  Process-wide; host only; always ILG_OK. */
ilg_status ilg_inject_alloc_failure(int64_t after);

#ifdef __cplusplus
}
#endif

#endif /* ILG_H */
