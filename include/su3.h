/*
 * su3.h -- C ABI of libsu3gb300: the checkerboard Cabibbo-Marinari heatbath
 * of pure SU(3) Wilson-action lattice gauge theory on one GB300 GPU
 * (sm_103a), after B. A. Berg, "Fortran MPI Checkerboard Code for SU(3)
 * Lattice Gauge Theory I" (arXiv:0904.0642).
 *
 * Conventions shared by every call
 * ---------------------------------
 * - Geometry (Sec. 2, eqs. i_s, xD, x^i, i_c): D directions, extents
 *   n^1..n^D (all even: the checkerboard needs it), site number
 *   i_s - 1 = sum_i x^i n_a^i with x^1 running fastest, colour
 *   mod(sum_i x^i, 2).  Direction D is time.
 * - Boundary (Sec. 2.2): SU3_PBC is the torus.  SU3_DLT is the
 *   double-layered torus: two identical lattices (layers 0 and 1); a step
 *   across the boundary of a glued direction lands on the other layer.
 * - Action (Sec. 2.1, Table 2): weight exp((beta/3) sum_p Re Tr U_p),
 *   beta = 6/g^2.
 * - Canonical host layout of links: double U[layer][site][mu][row][col][re,im]
 *   (18 doubles per link; D*V*layers links).  Device storage is internal.
 * - Random numbers: Philox4x32-10 with key = seed and counter
 *   (site key, sweep, tag(colour, mu, subgroup, hit), purpose), so every
 *   result is a deterministic function of (configuration, seed, sweep
 *   counter) and does not depend on launch shape, batching or graph use.
 * - Errors: every call returns an su3_status; nothing throws across the
 *   ABI.  On error, su3_last_error() returns a message (thread-local).
 * - Streams: a handle runs all its work on the cudaStream_t given at
 *   creation (NULL: a stream the library creates and owns; graphs
 *   cannot capture the legacy default stream).  Calls that return host
 *   values synchronise that stream; the others are asynchronous.
 * - Ownership: handles are owned by the caller and freed with the matching
 *   destroy call.  A caller-owned link buffer must outlive its handle.
 */
#ifndef SU3_GB300_H
#define SU3_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SU3_OK = 0,
  SU3_EINVAL = -1,    /* invalid argument (odd extent, D out of range, beta < 0, hits < 1, ...) */
  SU3_ENOMEM = -2,    /* device allocation failed or HBM budget exceeded */
  SU3_ECUDA = -3,     /* a CUDA runtime call failed */
  SU3_ETIMEOUT = -4,  /* a bounded wait ran out */
  SU3_EBUSY = -5,     /* result not ready yet */
  SU3_ENOTFOUND = -6  /* unknown job id */
} su3_status;

typedef enum { SU3_PBC = 0, SU3_DLT = 1 } su3_boundary;

/* Device link storage.  FP64_18: all 18 reals in double (144 bytes per
 * link).  FP32_12: the first two rows in float, the third rebuilt as
 * conj(row1 x row2) on load (48 bytes).  FP32_18: all 18 reals in float
 * (72 bytes; the third row is loaded, not rebuilt, and is renewed by
 * re-unitarisation).  Both float forms draw and update in float (Sec. 2.1:
 * the FHKP draw switches to double for alpha >= 32). */
typedef enum { SU3_FP64_18 = 0, SU3_FP32_12 = 1, SU3_FP32_18 = 2 } su3_storage;

typedef enum { SU3_START_COLD = 0, SU3_START_HOT = 1 } su3_start;

#define SU3_MAX_D 4 /* GPU kernels are compiled for D = 2, 3, 4 */

typedef struct su3_config {
  int32_t D;                    /* 2..SU3_MAX_D */
  int32_t dims[SU3_MAX_D];      /* n^1..n^D, even, >= 2 */
  int32_t boundary;             /* su3_boundary */
  int32_t glue_mask;            /* DLT: bit mu glues direction mu; 0 means all directions */
  double beta;                  /* >= 0 */
  uint64_t seed;                /* Philox key */
  int32_t storage;              /* su3_storage */
  int32_t start;                /* su3_start: ordered (all links 1) or Haar-random (Sec. 2.4, istart) */
  int32_t hits;                 /* FHKP proposals per SU(2) subgroup (Sec. 2.1, nhit), >= 1 */
  int32_t reunit_every;         /* re-unitarise every k sweeps inside su3_sweep (0: never) */
  int32_t measure_every;        /* record plaquette + Polyakov loop every k sweeps (0: never) */
  int32_t measure_capacity;     /* ring size of recorded measurements (0: 1024) */
  int32_t layer_blind;          /* DLT: identical random numbers on both layers (Sec. 3.2, lat2test) */
  int32_t rng_period[SU3_MAX_D];/* random-number site key uses x^i mod period (0: n^i); Sec. 3.1.1 test */
  void *stream;                 /* cudaStream_t, or NULL */
  void *link_buffer;            /* optional caller-owned device buffer for the links, or NULL */
  size_t link_buffer_bytes;     /* its size; must be >= su3_link_bytes() */
  double beta1;                 /* DLT with two couplings (Sec. 2.2): beta of the plaquettes with a link in
                                   layer 1; < 0 (the default of su3_config_init): equal to beta */
  int32_t ndiv[SU3_MAX_D];      /* sublattices per direction (the paper's MPI sublattices, Sec. 2.4, run on
                                   one device); 0 or 1: undivided.  See su3_lattice_create_ex. */
} su3_config;

typedef struct su3_lattice su3_lattice;

/* Fill *cfg with defaults: D=4, 4^4, PBC, beta=6 (beta1 = beta), seed=1,
 * FP64_18, cold, hits=2, no automatic re-unitarisation or measurement. */
void su3_config_init(su3_config *cfg);

/* Device bytes the links of cfg need (0 if cfg is invalid); for a divided
 * lattice (ndiv) the sublattice boxes plus the undivided copy. */
size_t su3_link_bytes(const su3_config *cfg);

/* Create a lattice: torus or DLT of the given extents, cold start, FP64_18
 * storage, beta, seed.  Validation as for su3_lattice_create_ex.  *out is
 * NULL on error. */
su3_status su3_lattice_create(int D, const int *dims, su3_boundary boundary, double beta, uint64_t seed,
                              su3_lattice **out);

/* Create a lattice from a full configuration.  EINVAL when D is outside
 * 2..SU3_MAX_D, an extent is odd or < 2, beta < 0, hits < 1, a period does
 * not divide its extent (or is odd), or the caller buffer is too small;
 * ENOMEM when the device allocation fails.  The start configuration is
 * written before return (asynchronously on the stream).
 *
 * Sublattice decomposition (ndiv[i] > 1 for some i; Sec. 2.4): the lattice
 * is cut into ndiv[i] sublattices along direction i, each of interior
 * extent n^i / ndiv[i] (even, >= 2, else EINVAL).  Every sublattice keeps
 * its links in its own box with one halo layer on both sides of each cut
 * direction; after every tick that changes links a halo kernel copies the
 * changed links (faces, and the corner links when two or more directions
 * are cut) from the sublattice that owns them.  The random numbers are
 * keyed by the undivided site, so results are bitwise those of the
 * undivided lattice.  Not with a caller-owned link buffer, ensembles or
 * the server, nor with two couplings on a DLT cut along a glued direction
 * (EINVAL).  The launch variant is fixed (su3_set_launch picks threads and
 * CTAs only); measurements recorded by measure_every hold NaN Polyakov
 * loops when the time direction is cut (su3_polyakov is exact in every
 * case: it reads the undivided layout).  su3_lattice_info reports the
 * bytes of the boxes; an undivided copy of the links is kept besides. */
su3_status su3_lattice_create_ex(const su3_config *cfg, su3_lattice **out);

/* Release the handle and its device memory (not a caller-owned buffer). */
void su3_lattice_destroy(su3_lattice *lat);

/* n checkerboard sweeps (Sec. 2.1: every link updated once, colour by
 * colour, direction by direction), each link by Cabibbo-Marinari over the
 * SU(2) subgroups (1,2), (1,3), (2,3) with the multi-hit FHKP heatbath
 * (`hits` proposals, the subgroup kept when none is accepted).  Honours
 * reunit_every and measure_every.  Asynchronous.  EINVAL for n < 0 or
 * hits < 1. */
su3_status su3_sweep(su3_lattice *lat, int n, int hits);

/* Re-unitarise every link (Sec. 2.4, su3reunit): Gram-Schmidt of rows 1, 2
 * in double precision, row 3 = conj(row1 x row2).  Asynchronous. */
su3_status su3_reunitarize(su3_lattice *lat);

/* Plaquette averages (Sec. 2.4 wloops, Table 2): (1/3) Re Tr U_p over the
 * plaquettes whose base site is in `layer` (layer = -1: the whole lattice),
 * total, space-like and time-like (time-like planes contain direction D;
 * *space is 0 when D = 2).  Double-precision accumulation with a fixed
 * reduction order.  Synchronises the stream.  Output pointers are host
 * pointers and may be NULL. */
su3_status su3_plaquette(su3_lattice *lat, int layer, double *total, double *space, double *time);

/* Polyakov loop: (1/3) Tr of the ordered product of U_D along the closed
 * line through (layer, x, x^D = 0) (length n^D, or 2 n^D on a DLT glued in
 * time), averaged over the spatial sites of the layer (-1: all layers).
 * Synchronises the stream.  Not in the paper. */
su3_status su3_polyakov(su3_lattice *lat, int layer, double *re, double *im);

/* Asynchronous measurement into device memory: writes 5 doubles per layer
 * slot, slots 0..layers-1 then the whole lattice, as
 * [total, space, time, poly_re, poly_im], to the device pointer out. */
su3_status su3_measure_async(su3_lattice *lat, double *device_out);

/* Measurements recorded by measure_every, oldest first: up to max entries
 * of 5*(layers+1) doubles each (layout as su3_measure_async) copied to the
 * host buffer; *count receives the number copied.  Synchronises. */
su3_status su3_measurements(su3_lattice *lat, double *host_out, size_t max, size_t *count);

/* The most recent of those recorded measurements only: 5*(layers+1)
 * doubles (n must hold them).  ENOTFOUND when none was recorded yet.
 * Synchronises. */
su3_status su3_measurement_latest(su3_lattice *lat, double *host_out, size_t n);

/* The same without waiting: queues the copy of the most recent measurement
 * recorded by the work queued so far (stream order) into host_out and
 * returns at once; ENOTFOUND when the queued sweeps record none.  host_out
 * should be page-locked (else the copy is not asynchronous) and is valid
 * once the lattice's stream has reached the copy: after su3_synchronize,
 * or an event the caller records on the stream it passed at creation.  A
 * pipelined caller reads step k's result while step k+1 runs. */
su3_status su3_measurement_latest_async(su3_lattice *lat, double *host_out, size_t n);

/* Wait until all work queued on the lattice's stream has finished.  In a
 * debug-bounds build also SU3_ECUDA when a device bounds check has failed
 * (see su3_bounds_status). */
su3_status su3_synchronize(su3_lattice *lat);

/* The same with a deadline (a host-side watchdog): polls an event recorded
 * behind the queued work and returns SU3_ETIMEOUT once timeout_s seconds
 * have passed; the work keeps running and a later call can wait again.
 * EINVAL for a negative timeout. */
su3_status su3_wait(su3_lattice *lat, double timeout_s);

/* Copy all links to / from the host in the canonical layout; n is the
 * number of doubles in the host buffer (>= 18 * links).  set_links rounds
 * to the storage precision (FP32_12 keeps rows 1 and 2, FP32_18 rounds all
 * 18 reals to float).  Synchronous. */
su3_status su3_get_links(su3_lattice *lat, double *host, size_t n);
su3_status su3_set_links(su3_lattice *lat, const double *host, size_t n);

/* Asynchronous link input, for inputs that arrive while the lattice is
 * sweeping.  su3_stage_links starts the copy of n >= links*18 doubles
 * (canonical layout, as su3_set_links) from host memory into one of two
 * device staging buffers on the library's own copy stream and returns at
 * once; with pinned host memory the copy overlaps the sweeps already
 * queued.  At most one staged input may wait: EBUSY until su3_apply_links.
 * su3_apply_links makes the lattice's stream wait for that copy, then
 * converts the staged links into the lattice (divided lattices: scatter and
 * halo refresh) and restarts the action bookkeeping, all queued on the
 * stream without blocking the host; EINVAL when nothing is staged.  With
 * measure_every > 0 (one coupling) the bookkeeping restarts at the next
 * recorded measurement, which measures the action anyway, instead of with a
 * measurement of its own (su3_action before then restarts it on the spot).  The
 * host buffer is read asynchronously: keep it unchanged until a
 * synchronising call on the lattice (su3_plaquette, su3_get_links, ...)
 * has returned after the matching su3_apply_links. */
su3_status su3_stage_links(su3_lattice *lat, const double *host, size_t n);
su3_status su3_apply_links(su3_lattice *lat);

/* su3_stage_links with a choice of host format: SU3_LINKS_FP64_18 (as
 * su3_stage_links: n >= links*18 doubles) or SU3_LINKS_FP32_12 (rows 1 and
 * 2 of every link as floats, [layer][i_s-1][mu][row 1..2][col][re,im], so
 * n >= links*12 floats, 16-byte aligned; row 3 is rebuilt as
 * conj(row1 x row2) -- the two-row form of the FP32_12 storage, a third of
 * the bytes of the canonical layout). */
typedef enum { SU3_LINKS_FP64_18 = 0, SU3_LINKS_FP32_12 = 1 } su3_links_format;
su3_status su3_stage_links_ex(su3_lattice *lat, const void *host, size_t n, int format);

/* Counters: FHKP proposals and accepted proposals since creation, and the
 * number of completed sweeps (the sweep counter of the random numbers). */
su3_status su3_stats(su3_lattice *lat, uint64_t *proposals, uint64_t *accepts, uint64_t *sweeps);

/* Action bookkeeping (Sec. 2.1: the update keeps track of the total action,
 * checked now and then against a direct recalculation).  Every link update
 * books its change of S = sum_p beta_p (1 - Re Tr U_p / 3): an accepted SU(2)
 * subgroup changes Re Tr(U A) by 2 (k x0 - a0).  *booked = the action at the
 * last reset + the booked changes since (summed in a fixed order); *direct =
 * the action recomputed from the plaquette now (NaN for the two-coupling DLT;
 * its *booked is then the change since the last reset).  Re-unitarisation
 * and su3_set_links are not booked; su3_set_links resets (su3_apply_links
 * too, possibly at the next recorded measurement).  Synchronises.
 * su3_action_reset sets the reference to the direct action and clears the
 * booked changes. */
su3_status su3_action(su3_lattice *lat, double *booked, double *direct);
su3_status su3_action_reset(su3_lattice *lat);

/* Set the sweep counter (resume from a checkpoint taken with su3_get_links
 * and su3_stats: the counter-based random numbers make the continuation
 * bitwise identical). */
su3_status su3_set_sweep_counter(su3_lattice *lat, uint64_t sweeps);

/* Number of links (D*V*layers) and device bytes of the link storage. */
su3_status su3_lattice_info(su3_lattice *lat, size_t *links, size_t *bytes);

/* Launch shape.  variant: register variant of the update kernel (FP32_12
 * storage: 0 = 128 registers / up to 256 threads, 1 = 96 / up to 128,
 * 2 = 96 / up to 128, 3 = 128 / up to 256 and 4 = 85 / up to 256 with the
 * loop over staple directions kept rolled; FP32_18 and FP64 storage: 0
 * only).  threads:
 * CTA width, a multiple of 32 up to the variant's maximum.  ctas_per_sm = 0
 * launches one CTA per tile of `threads` sites; > 0 a persistent grid of
 * (SM count x ctas_per_sm) CTAs that loop over the tiles.  The random
 * numbers do not depend on the shape, so results are identical for every
 * choice.  su3_autotune times the candidates on this lattice, each from the
 * same links (links, counters and sweep counter are restored afterwards),
 * and keeps the fastest; outputs may be NULL. */
su3_status su3_set_launch(su3_lattice *lat, int variant, int threads, int ctas_per_sm);
su3_status su3_autotune(su3_lattice *lat, int *variant, int *threads, int *ctas_per_sm, double *us_per_sweep);

/* Capture the sweep in a CUDA graph (on = 1) or launch kernel by kernel
 * (on = 0).  Results are identical either way. */
su3_status su3_use_graph(su3_lattice *lat, int on);

/* Launch each update tick as a programmatic dependent of the previous one
 * (on by default): the next tick is scheduled while the previous one ends
 * and waits at its first instruction for the previous tick's completion
 * and memory, so results are identical either way.  Where the driver
 * refuses such launches the library falls back to ordinary ones. */
su3_status su3_use_pdl(su3_lattice *lat, int on);

/* Kernel timing.  With profiling on, su3_sweep launches its ticks one by
 * one (no graph) with a CUDA event pair around each on the handle's stream,
 * and su3_get_profile sums the device time per stage kind: update phases,
 * re-unitarisations, measurements (synchronises; reset = 1 clears).  The
 * results do not change. */
typedef struct su3_profile {
  double update_ms;
  int64_t update_launches;
  double reunit_ms;
  int64_t reunit_launches;
  double measure_ms;
  int64_t measure_launches;
} su3_profile;

su3_status su3_set_profiling(su3_lattice *lat, int on);
su3_status su3_get_profile(su3_lattice *lat, su3_profile *out, int reset);

/* ---------------------------------------------------------------- measurement without allocation
 * The paper has no counterpart to this call; it exists for users of the
 * library.
 *
 * su3_measure_noalloc computes what su3_measure_async computes (plaquette
 * total / space / time and Polyakov loop, per layer and for the whole
 * lattice) for links the caller already holds on the device, and allocates
 * no memory at all, device or host.  It is for callers that cannot call
 * cudaMalloc: code embedded in a host framework whose memory pool must stay
 * the only owner of device memory, loops that cannot take the device-wide
 * synchronisation an allocation may cause, and plug-ins that run under a
 * fixed device-memory budget.
 *
 * cfg:        geometry and storage of the links (D, dims, boundary,
 *             glue_mask, storage): only these fields are read and
 *             validated; every other field is ignored (a zero-filled
 *             struct with these five set is accepted).
 * links:      device pointer to link storage in the library's layout,
 *             16-byte aligned (e.g. the caller-owned link_buffer a lattice
 *             was created with).
 * device_out: device pointer to 5*(layers+1) doubles, written as
 *             [total, space, time, poly_re, poly_im] for each layer, then for
 *             the whole lattice.
 * stream:     cudaStream_t (NULL: the legacy default stream); asynchronous.
 *
 * Scratch: the per-block partial sums go to a fixed 1 MiB array inside the
 * library (32768 slots), which every GPU that loads the library holds until
 * the process exits.  A lattice needs one slot per tile of 256 sites of one
 * colour in each layer: layers x ceil(V / 2 / 256) slots, V the sites of one
 * layer (each layer's count is rounded up to whole tiles).  A lattice that
 * needs more than 32768 slots (64^4 PBC needs exactly 32768) is rejected
 * with SU3_EINVAL before anything is launched.  Each call writes every slot
 * it reads, so nothing needs clearing between calls, but all calls share
 * the one array: calls that overlap on the GPU (other streams, other
 * threads) race, so serialise them.
 * Set-up: the first call on each device looks up the device address of the
 * array (cudaGetSymbolAddress) and keeps it with the id of the current
 * context; a later call in another context of that device (after
 * cudaDeviceReset, say) looks it up again.  Make the first call on a
 * device, and the first after a reset, before any stream capture. */
su3_status su3_measure_noalloc(const su3_config *cfg, const void *links, double *device_out, void *stream);

/* ---------------------------------------------------------------- ensembles
 * Many independent chains (each with its own extents, boundary, beta, seed
 * and hits; one storage for all) advanced together: one fused persistent
 * launch per checkerboard phase covers every chain.  A chain gives the same
 * links in an ensemble as alone, bit for bit. */
typedef struct su3_ensemble su3_ensemble;

su3_status su3_ensemble_create(const su3_config *cfgs, int nchains, void *stream, su3_ensemble **out);
void su3_ensemble_destroy(su3_ensemble *ens);
/* n sweeps of every chain (hits from each config). */
su3_status su3_ensemble_sweep(su3_ensemble *ens, int n);
/* su3_wait for an ensemble: the queued work, with a deadline (ETIMEOUT). */
su3_status su3_ensemble_wait(su3_ensemble *ens, double timeout_s);
/* Plaquette and Polyakov loop of every chain, whole lattice: out[5*c + k],
 * k = total, space, time, poly_re, poly_im.  Synchronises. */
su3_status su3_ensemble_measure(su3_ensemble *ens, double *host_out);
su3_status su3_ensemble_get_links(su3_ensemble *ens, int chain, double *host, size_t n);
/* As su3_measurements, for one chain of the ensemble (its measure_every). */
su3_status su3_ensemble_measurements(su3_ensemble *ens, int chain, double *host_out, size_t max, size_t *count);
su3_status su3_ensemble_set_launch(su3_ensemble *ens, int variant, int threads, int ctas_per_sm);
su3_status su3_ensemble_autotune(su3_ensemble *ens, int *variant, int *threads, int *ctas_per_sm,
                                 double *us_per_sweep);
su3_status su3_ensemble_use_graph(su3_ensemble *ens, int on);
/* As su3_set_profiling / su3_get_profile; stages are classified by chain 0. */
su3_status su3_ensemble_set_profiling(su3_ensemble *ens, int on);
su3_status su3_ensemble_get_profile(su3_ensemble *ens, su3_profile *out, int reset);

/* ---------------------------------------------------------------- serving
 * A job server with continuous batching: submitted jobs wait in a queue,
 * are admitted when a slot and enough of the HBM budget are free, run
 * together in the fused launch (each chain at its own phase), and retire
 * when their sweeps are done, which frees memory for the queue. */
typedef struct su3_server su3_server;

typedef struct su3_job {
  su3_config cfg;          /* lattice of the job (stream and link_buffer ignored) */
  int32_t sweeps;          /* sweeps to run, >= 1 */
  /* Optional host buffers (NULL: unused), each layers*V*D*18 doubles in the
   * canonical layout of su3_get_links, owned by the caller and read or
   * written by the server's worker thread: they must stay valid until the
   * job's result has been collected (su3_server_poll / su3_server_wait).
   * links_in:  start configuration, replacing cfg.start (written at
   *            admission, as su3_set_links would).
   * links_out: receives the links after the last sweep, at retirement. */
  const double *links_in;
  double *links_out;
} su3_job;

typedef struct su3_result {
  uint64_t job_id;
  int32_t status;          /* su3_status of the job */
  int32_t nlayers;
  double plaquette[3];     /* whole lattice after the last sweep: total, space, time */
  double polyakov[2];
  double layer_plaquette[2];  /* per layer, total */
  uint64_t proposals, accepts;
  double submit_s, start_s, finish_s;  /* host clock (seconds since server creation) */
} su3_result;

/* hbm_budget_bytes: device bytes the resident chains may hold (0: 80 % of
 * free memory); max_slots: resident chains at most.
 * The worker thread runs the resident chains in rounds of 16 fused ticks
 * (one captured graph) and reads their stage machines back after each
 * round (one host synchronisation per round): admission and retirement
 * happen between rounds, which sets the granularity of job latency. */
su3_status su3_server_create(size_t hbm_budget_bytes, int max_slots, su3_server **out);
/* Queue a job; never blocks.  EINVAL for a bad job, ENOMEM when the job
 * alone exceeds the budget, ECUDA (with the worker's message) once the
 * worker has stopped after an error. */
su3_status su3_server_submit(su3_server *srv, const su3_job *job, uint64_t *job_id);
/* EBUSY while queued or running, OK with *out filled once done, ENOTFOUND
 * for an unknown (or already collected) id.  A job that fails on its own
 * (its device allocation at admission, its measurement) is done with that
 * status in out->status.  When the worker itself has stopped after an
 * error (a failed launch or synchronisation), every job not yet done gets
 * ECUDA with the worker's message from poll and wait, instead of EBUSY or
 * a timeout. */
su3_status su3_server_poll(su3_server *srv, uint64_t job_id, su3_result *out);
su3_status su3_server_wait(su3_server *srv, uint64_t job_id, double timeout_s, su3_result *out);
/* Jobs queued, resident, and finished-but-uncollected. */
su3_status su3_server_load(su3_server *srv, int *queued, int *resident, int *finished);
/* Rounds of fused ticks the worker has run and their device time in
 * milliseconds (CUDA events around each round on the worker's stream: the
 * kernels of the rounds, without the host work between rounds). */
su3_status su3_server_stats(su3_server *srv, uint64_t *rounds, double *device_ms);
/* Stops the scheduler; jobs still queued or running end with SU3_EBUSY. */
void su3_server_destroy(su3_server *srv);

/* ---------------------------------------------------------------- fault injection
 * For tests of the error paths, on the host only (no GPU fault is ever
 * caused): arm the next `count` passes through `site` to fail as the real
 * failure would (count 0 disarms).  Sites:
 *   "server_admit"  the admission of a job fails as its device allocation
 *                   would (that job is done with SU3_ENOMEM; the worker
 *                   carries on);
 *   "server_round"  the worker's next round of ticks fails as a failed
 *                   launch would (the worker stops; see su3_server_poll).
 * EINVAL for an unknown site or a negative count. */
su3_status su3_inject_fault(const char *site, int count);

/* ---------------------------------------------------------------- debug bounds checks
 * A library built with SU3_DEBUG_BOUNDS (libsu3gb300_dbg.so, built beside
 * the release library) checks every link access and every scratch index on
 * the device against its extent before the access.  The first violation is
 * recorded in device memory and the access is skipped; nothing traps, so
 * the context stays usable.  su3_synchronize then returns SU3_ECUDA with the
 * violation in su3_last_error.  The release library compiles the checks
 * out: there su3_bounds_status always reports none.
 *
 * su3_bounds_status: the first recorded violation (site code, index,
 *   extent; site 0: none); SU3_OK when none, SU3_ECUDA otherwise.  The
 *   record is sticky for the life of the process.  Synchronises the device.
 * su3_bounds_selftest: records a deliberate violation (an index equal to
 *   its extent, checked but never used for an access) to test the reporting
 *   path; SU3_EINVAL in the release library. */
su3_status su3_bounds_status(uint64_t *site, int64_t *index, int64_t *extent);
su3_status su3_bounds_selftest(void);

/* Thread-local message of the last error (empty string if none). */
const char *su3_last_error(void);
/* Library version string. */
const char *su3_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SU3_GB300_H */
