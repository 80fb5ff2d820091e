/*
 * isg.h -- C ABI of libisg: the checkerboard single-spin-flip Metropolis sweep
 * of the 2D spin-1/2 Ising and spin-1 Blume-Capel models on an L x L periodic
 * square lattice, on one NVIDIA B300 (sm_103a), with the per-sweep
 * observables behind the energy, the magnetisation and the second-moment
 * correlation length.
 *
 * Model (Eq. (1) of arXiv 2503.14688):
 *     H = -J sum_<xy> s_x s_y + Delta sum_x s_x^2,   J = 1,
 *     s in {-1,+1} (Ising) or {-1,0,+1} (Blume-Capel).
 * Dynamics (Introduction; Table I): Metropolis, made parallel by a
 * checkerboard decomposition; the unit of time is one full-lattice sweep.
 * Random numbers (Appendix B): 32-bit integers, here Philox4x32-10 keyed per
 * site, so every accept/reject is an integer comparison and every result is
 * reproducible bit for bit.
 *
 * Conventions used by every call:
 *   - Site (x, y), x, y in [0, L); colour c = (x + y) & 1; same-colour index
 *     j = (y*L + x) >> 1.  Sweep t updates colour 0, then colour 1, both with
 *     the inverse temperature beta(t).
 *   - Random word of a site at sweep t: word (j & 3) of Philox4x32-10 with
 *     key (lo32(seed), hi32(seed)) and counter (lo32(j>>2), hi32(j>>2), t, c).
 *     The hot start uses the counter (lo32(j>>2), hi32(j>>2), 0, c | 2).
 *   - Acceptance of a move with energy change dE: always if dE <= 0; else
 *     Ising iff u < rne(2^32 exp(-beta dE)), Blume-Capel iff
 *     (u >> 1) < rne(2^31 exp(-beta dE)), with the thresholds computed on the
 *     host in FP64 (libm exp, round to nearest even).
 *   - Blume-Capel proposal: bit b = u & 1 picks the new value as the (b+1)-th
 *     smallest of the two values different from the current one.
 *   - Valid L: a multiple of 64 (each colour row is a whole number of 32-bit
 *     words), 64 <= L <= 2^20 (Ising) or 2^19 (Blume-Capel), limited in
 *     practice by free device memory.  Sweep indices must stay below 2^32.
 *   - Every call returns an isg_status (0 = success) except the few that
 *     return a size, a double or a string; no C++ exception or abort crosses
 *     the ABI.  isg_last_error() gives a message for the calling thread.
 *   - Device work is queued on the stream given at creation and is
 *     asynchronous unless the call says it synchronises.  Calls on one
 *     object from several host threads at once are not supported.
 *   - The library owns the device memory it allocates.  The caller owns every
 *     host array it passes and any device buffer it lends (device_buf).
 *   - Without a usable CUDA device, the calls that need one return
 *     ISG_ERR_UNSUPPORTED; nothing falls back to the CPU.
 */
#ifndef ISG_H
#define ISG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t isg_status;
#define ISG_OK 0
#define ISG_ERR_INVALID (-1)        /* bad argument; nothing was queued           */
#define ISG_ERR_OOM (-2)            /* device (or pinned host) allocation failed  */
#define ISG_ERR_CUDA (-3)           /* a CUDA runtime call failed                 */
#define ISG_ERR_DEVICE_TIMEOUT (-4) /* a bounded device-side wait gave up         */
#define ISG_ERR_BUSY (-5)           /* no room (record ring full, server full)    */
#define ISG_ERR_UNSUPPORTED (-6)    /* no usable CUDA device                      */

#define ISG_ISING 0
#define ISG_BLUME_CAPEL 1

typedef struct isg_lattice isg_lattice;

/* Creation parameters of one lattice. */
typedef struct {
    int32_t model;           /* ISG_ISING or ISG_BLUME_CAPEL                      */
    int64_t L;               /* side; see "Valid L" above                         */
    uint64_t seed;           /* Philox key of this lattice                        */
    double delta;            /* crystal field Delta of Eq. (1); ignored for Ising */
    void *stream;            /* cudaStream_t for all work, NULL = default stream  */
    void *device_buf;        /* optional caller-owned device memory for the spins */
    size_t device_buf_bytes; /* its size; must be >= isg_lattice_bytes(model, L)  */
    int64_t record_capacity; /* observable records kept on the device (>= 1)      */
} isg_lattice_desc;

/* Observables of one lattice after one sweep (Eqs. (2)-(3); Appendix B).
 *   B = sum_x s_x (s_{x+e1} + s_{x+e2})   (bond sum; energy per spin is
 *                                          e = (-B + Delta Q) / L^2)
 *   M = sum_x s_x,  Q = sum_x s_x^2,
 *   row_sums[y] = sum_x s(x, y),  col_sums[x] = sum_y s(x, y).
 * row_sums / col_sums point to caller-owned HOST arrays of L int32 each (or
 * NULL to skip them). */
typedef struct {
    int64_t sweep; /* number of sweeps done when the record was taken         */
    int64_t B, M, Q;
    int32_t *row_sums;
    int32_t *col_sums;
} isg_obs;

/* A piecewise-constant bath: beta(t) = beta[i] for t_start[i] <= t <
 * t_start[i+1] (the last piece runs to the end).  t_start[0] must be <= the
 * first sweep index used and t_start must increase.  This is the paper's
 * time-dependent bath of the pre-cooling protocol ("Thermal protocols";
 * Table II: T1 until t_switch, then T2). */
typedef struct {
    int64_t n_pieces;
    const int64_t *t_start;
    const double *beta;
} isg_schedule;

/* Bytes of device memory the spins of an L x L lattice occupy: L^2/8 for
 * Ising (1 bit per site), L^2/4 for Blume-Capel (2 bit-planes).  0 if the
 * model or L is invalid. */
size_t isg_lattice_bytes(int32_t model, int64_t L);

/* Create a lattice on the current CUDA device.  Allocates the spin planes
 * (unless desc->device_buf is given) and the record ring (record_capacity
 * records of 32 + 8 L bytes).  The spins are undefined until an init or set
 * call.  *out is NULL on failure. */
isg_status isg_lattice_create(const isg_lattice_desc *desc, isg_lattice **out);

/* Release everything the lattice owns (waits for its stream first).  NULL is
 * accepted. */
void isg_lattice_destroy(isg_lattice *lat);

/* Hot start ("Thermal protocols": the direct quench starts from T = infinity,
 * a fully disordered configuration): Ising s = +1 iff u >= 2^31,
 * Blume-Capel s = ((3 u) >> 32) - 1, u the site's hot-start random word.
 * Resets the sweep counter to 0 and drops pending records. */
isg_status isg_lattice_init_random(isg_lattice *lat);

/* Cold start: every site = value (+1/-1; also 0 for Blume-Capel).  Resets
 * the sweep counter to 0 and drops pending records. */
isg_status isg_lattice_init_uniform(isg_lattice *lat, int8_t value);

/* Load L*L host bytes (row-major, s[y*L + x]) and set the sweep counter to
 * t.  Synchronises.  ISG_ERR_INVALID on a value outside the model's set. */
isg_status isg_lattice_set(isg_lattice *lat, const int8_t *host, int64_t t);

/* Copy the h x w window with corner (y0, x0), periodic wrap, to host bytes
 * out[i*w + j] = s(x0 + j, y0 + i).  Synchronises. */
isg_status isg_lattice_get_rect(isg_lattice *lat, int64_t y0, int64_t x0, int64_t h,
                                int64_t w, int8_t *out);

/* Whole lattice (L*L host bytes); the same as the rect with the full size. */
isg_status isg_lattice_get(isg_lattice *lat, int8_t *out);

/* Checkpoint: write the lattice to `path` -- a 64-byte header (magic
 * "ISGLAT01", int32 model, int32 0, int64 L, uint64 seed, double delta,
 * int64 sweep counter, uint64 plane bytes, 8 bytes 0), then the spin planes
 * exactly as stored on the device (little-endian 32-bit words).  Pending
 * records are not saved.  Synchronises; streams through a 64 MiB pinned
 * buffer, so lattices larger than host memory can be saved. */
isg_status isg_save(isg_lattice *lat, const char *path);

/* Resume: create a lattice (on the current device, work on `stream`, with
 * `record_capacity` record slots) from a file written by isg_save.  Sweeping
 * it continues the run bit for bit (the random numbers depend only on seed,
 * sweep index, colour and site).  ISG_ERR_INVALID for a missing, short or
 * foreign file.  Synchronises. */
isg_status isg_load(const char *path, void *stream, int64_t record_capacity, isg_lattice **out);

/* Sweep counter (sweeps done so far), L, model, seed. */
isg_status isg_lattice_info(const isg_lattice *lat, int64_t *sweep, int64_t *L,
                            int32_t *model, uint64_t *seed);

/* Run n Metropolis sweeps t0 .. t0+n-1 (t0 = the sweep counter), sweep t0+i
 * at inverse temperature betas[i] (betas: n host doubles) or beta_const when
 * betas is NULL.  beta must be >= 0 (+inf allowed: only dE <= 0 moves).
 * With record_every = k > 0, the observables after every k-th sweep of this
 * call are appended to the record ring; ISG_ERR_BUSY (nothing queued) if the
 * ring has too little room.  Asynchronous. */
isg_status isg_sweep(isg_lattice *lat, int64_t n, const double *betas, double beta_const,
                     int64_t record_every);

/* The same with beta(t) from a piecewise-constant schedule. */
isg_status isg_sweep_schedule(isg_lattice *lat, int64_t n, const isg_schedule *sched,
                              int64_t record_every);

/* One half of the current sweep: colour 0 or 1 at inverse temperature beta.
 * Colour 1 completes the sweep and advances the counter.  For timing a
 * single kernel; isg_sweep is the normal entry. */
isg_status isg_half_sweep(isg_lattice *lat, int32_t colour, double beta);

/* Append the observables of the current lattice to the record ring.
 * Asynchronous.  ISG_ERR_BUSY if the ring is full. */
isg_status isg_record(isg_lattice *lat);

/* Move up to max pending records, oldest first, into out[0..]: the scalars,
 * and the row/column sums into the host arrays each out[i] points to (if not
 * NULL).  *count = records moved.  Synchronises.  A record whose pass ran
 * out of time (a bounded wait of the streamed record pass gave up) is
 * dropped from the ring and the call returns ISG_ERR_DEVICE_TIMEOUT with
 * *count = the records moved before it. */
isg_status isg_read_records(isg_lattice *lat, isg_obs *out, int64_t max, int64_t *count);

/* Number of records waiting in the ring. */
isg_status isg_pending_records(const isg_lattice *lat, int64_t *count);

/* Observables of the current lattice into *out (host arrays).  Does not touch
 * the record ring.  Synchronises.  ISG_ERR_DEVICE_TIMEOUT if the record
 * pass ran out of time (a bounded wait gave up; see ISG_INJECT_WAIT). */
isg_status isg_measure(isg_lattice *lat, isg_obs *out);

/* Largest L accepted by isg_measure_planes_noalloc. */
#define ISG_NOALLOC_MAX_L ((int64_t)1 << 18)

/* The paper has no counterpart of this call: it serves callers that cannot
 * allocate device memory when they measure -- a process whose device memory
 * is all handed out by its own pool allocator, or a loop running many
 * lattices on concurrent streams that cannot afford the device-wide
 * synchronisation cudaMalloc/cudaFree may cause.
 *
 * Same observables as isg_measure (B, M, Q and, if the out pointers are not
 * NULL, the row/column sums into caller HOST arrays of L int32 each), for
 * spin planes held in caller memory: d_planes is a device pointer to
 * isg_lattice_bytes(model, L) bytes in the plane layout that a lattice
 * created with that buffer as device_buf keeps there (16-byte aligned, read
 * only).  out->sweep is set to `sweep` (a label of the caller's choosing).
 * Work is queued on `stream` (NULL = default stream) and the call waits for
 * that stream before returning.
 *
 * Allocates nothing: it accumulates into one fixed array of 32 + 8 L bytes
 * for L <= ISG_NOALLOC_MAX_L (2 MiB + 32 bytes) in the library's device
 * image, which every GPU that loads the library holds until the process
 * exits.  L above that limit is rejected with ISG_ERR_INVALID (use
 * isg_measure).  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it for
 * the life of the process; make that first call before any stream capture,
 * and do not reset the device (cudaDeviceReset) while the library is
 * loaded, since the kept address would then be stale.  Each call clears the part of the array it
 * uses before accumulating.  All calls on one device share the array: calls
 * whose GPU work overlaps (for instance from two host threads on two
 * streams) race on it and their results are undefined; calls made one after
 * another never overlap, since each waits for its stream, on failure too. */
isg_status isg_measure_planes_noalloc(int32_t model, int64_t L, const void *d_planes,
                                      void *stream, int64_t sweep, isg_obs *out);

/* Second-moment correlation length of Appendix B for an ensemble of n
 * lattices of side L, from their M[r] and row/column sums R[r*L + y],
 * C[r*L + x] (host arrays):
 *   S0 = M^2 (exact), Sk = (|M(2pi/L,0)|^2 + |M(0,2pi/L)|^2) / 2,
 *   xi2 = sqrt(<S0>/<Sk> - 1) / (2 sin(pi/L)),
 * replica averages taken first.  Host FP64 in a fixed operation order
 * (twiddles from libm on the first octant and exact symmetries, compensated
 * sums in index order), so equal integers give equal bits.  NaN if
 * <S0> <= <Sk> or an argument is invalid; +inf if <Sk> = 0 < <S0>. */
double isg_xi2(int64_t n, int64_t L, const int64_t *M, const int32_t *R, const int32_t *C);

/* ---------------------------------------------------------------------------
 * Ensembles: many independent replicas (the replica averages of Eqs. (2)-(3)
 * and Appendix B), of uneven L and models, swept together.  Replicas that fit
 * in shared memory (Ising L <= 1280, Blume-Capel L <= 896) are run by one
 * persistent kernel -- each CTA takes whole replicas from a work counter,
 * largest first, and keeps them in shared memory for all sweeps of a call;
 * larger replicas are grouped by (model, L) and each group is swept by
 * multi-lattice launches (up to 240 lattices each) on the same stream.
 * Replica r evolves bit for bit like a lattice created alone with seed[r].
 * ------------------------------------------------------------------------- */
typedef struct isg_ensemble isg_ensemble;

typedef struct {
    int64_t n;               /* number of replicas (>= 1)                        */
    const int64_t *L;        /* n sides (valid L as for lattices)                */
    const int32_t *model;    /* n models, or NULL for all Ising                  */
    const uint64_t *seed;    /* n Philox keys                                    */
    double delta;            /* Blume-Capel crystal field, shared                */
    void *stream;            /* cudaStream_t; NULL = an internal stream          */
    int64_t record_capacity; /* record rows kept on the device (>= 1); a row
                                holds one record per replica (32 + 8 L_r bytes) */
} isg_ensemble_desc;

/* Allocate all replicas' planes and the record ring; spins undefined. */
isg_status isg_ensemble_create(const isg_ensemble_desc *desc, isg_ensemble **out);

/* Release everything (waits for the stream).  NULL is accepted. */
void isg_ensemble_destroy(isg_ensemble *ens);

/* Hot start of every replica (as isg_lattice_init_random with seed[r]);
 * sweep counter 0, records dropped. */
isg_status isg_ensemble_init_random(isg_ensemble *ens);

/* n sweeps of every replica at betas[i] (n host doubles) or beta_const; with
 * record_every = k > 0 one record row after every k-th sweep of the call
 * (ISG_ERR_BUSY if the ring lacks room).  The device work of the call (the
 * threshold upload, one persistent launch, the large replicas' launches) is
 * captured in a CUDA graph, instantiated once and updated in place by later
 * calls of the same shape; a call whose large replicas need more than 2^16
 * launches (2048 multi-lattice ones) is queued on the stream directly
 * instead.  Asynchronous. */
isg_status isg_ensemble_sweep(isg_ensemble *ens, int64_t n, const double *betas,
                              double beta_const, int64_t record_every);

/* Move up to `rows` oldest record rows into out[i*n + r] (replica r of row
 * i): scalars, and row/column sums into the host arrays out[] points to (if
 * not NULL; L_r int32 each).  *count = rows moved.  Synchronises. */
isg_status isg_ensemble_read_records(isg_ensemble *ens, int64_t rows, isg_obs *out,
                                     int64_t *count);

/* Replica r's lattice as L_r * L_r host bytes (row-major).  Synchronises. */
isg_status isg_ensemble_get(isg_ensemble *ens, int64_t r, int8_t *out);

/* Replicas, sweeps done, pending record rows, threads per CTA in use. */
isg_status isg_ensemble_info(const isg_ensemble *ens, int64_t *n, int64_t *sweep,
                             int64_t *pending, int32_t *threads_per_cta);

/* Launch shape of an ensemble's sweeps.  Part 0, the persistent
 * shared-memory kernel: threads per CTA (256, 512, 1024), whether replicas
 * that fit half the shared memory run on half-CTA teams, and how many sweeps
 * one launch covers (0: the whole call; else a call is cut into launches of
 * that many sweeps, rounded up to a multiple of record_every, at most 32).
 * Part 1, the multi-lattice launches of the replicas too large for shared
 * memory: words per thread (1, 2, 4) and rows per thread band (16, 32, 64);
 * 0 = chosen from L.  The results never depend on the shape. */
typedef struct {
    int32_t threads_per_cta;
    int32_t half_teams;
    int64_t sweeps_per_launch;
    int32_t multi_words;
    int32_t multi_band;
    double ms;     /* isg_ensemble_autotune: this candidate's time for its part */
    int32_t part;  /* isg_ensemble_autotune: 0 persistent kernel, 1 multi-lattice */
} isg_ensemble_tuning;

/* Choose the launch shape by timing `sweeps` sweeps (50 or more recommended)
 * of every candidate on a copy of the replicas (their state is not changed):
 * part 0 over 3 CTA sizes x teams on/off x {whole call, sweeps/5 per
 * launch}, part 1 over words {auto, 1, 2, 4} x bands {auto, 16, 32, 64}; the
 * fastest of each part is kept.  *best (may be NULL) = the choice, its ms the
 * sum of both parts' times; tried[0..min(max_tried, n))] (may be NULL when
 * max_tried is 0) = every candidate with its time, *n_tried = their number.
 * Synchronises. */
isg_status isg_ensemble_autotune(isg_ensemble *ens, int64_t sweeps, isg_ensemble_tuning *best,
                                 isg_ensemble_tuning *tried, int64_t max_tried, int64_t *n_tried);

/* Set or read the launch shape (ms and part ignored / 0).  ISG_ERR_INVALID
 * for a shape outside the ranges above.  Set synchronises. */
isg_status isg_ensemble_set_tuning(isg_ensemble *ens, const isg_ensemble_tuning *t);
isg_status isg_ensemble_get_tuning(const isg_ensemble *ens, isg_ensemble_tuning *t);

/* ---------------------------------------------------------------------------
 * Request server with continuous batching.  Each request is one lattice
 * (model, L, seed, Delta) run for n_sweeps sweeps under its own bath schedule
 * beta(t) -- the direct quench (one piece) or the time-dependent bath of the
 * pre-cooling protocol ("Thermal protocols"; Table II), or any stepped bath.
 * The server works in rounds (isg_server_step): it retires finished
 * requests, admits arrived requests in arrival order while the device-memory
 * budget and the slot count allow, and advances every running request by
 * chunk_sweeps sweeps -- lattices that fit in shared memory (Ising L <= 1280,
 * Blume-Capel L <= 896) together in one persistent launch, larger ones on
 * streams of their own, overlapping it.  Those streams carry priorities by
 * size (the largest lattices the least; the internal main stream the
 * greatest), so that mid-size requests' launches are scheduled ahead of the
 * largest ones' remaining blocks.  A result does not depend on what
 * else ran or where chunks were cut (per-site keying).  Requests leave the
 * schedule when done, when cancelled, when their deadline passes, or when
 * their allocation or a launch fails; each outcome is a state of
 * isg_result, and a failure never stops the others.
 * ------------------------------------------------------------------------- */
typedef struct isg_server isg_server;

#define ISG_REQ_QUEUED 0
#define ISG_REQ_RUNNING 1
#define ISG_REQ_DONE 2
#define ISG_REQ_CANCELLED 3  /* isg_server_cancel before it finished           */
#define ISG_REQ_EXPIRED 4    /* its deadline passed before it finished          */
#define ISG_REQ_FAILED 5     /* its allocation or a launch failed (error field) */

typedef struct {
    size_t hbm_budget;      /* device bytes requests may hold (capped at the free
                               memory at creation)                               */
    int32_t max_active;     /* requests resident at once (>= 1)                  */
    int64_t chunk_sweeps;   /* sweeps per request per round (>= 1)               */
    void *stream;           /* main stream; NULL = an internal stream            */
} isg_server_desc;

typedef struct {
    int32_t model;
    int64_t L;              /* a valid side (a multiple of 64)                   */
    uint64_t seed;
    double delta;           /* Blume-Capel crystal field                         */
    int64_t n_sweeps;       /* >= 1                                              */
    int64_t n_pieces;       /* beta(t) = beta[i] for t_start[i] <= t < t_start[i+1];
                               t_start[0] = 0, increasing; copied at submit      */
    const int64_t *t_start;
    const double *beta;
    int64_t record_every;   /* periodic records (0 = none); for requests batched
                               in shared memory it must divide chunk_sweeps      */
    int32_t keep_result;    /* 1: keep lattice and records until
                               isg_server_release; 0: free them when done        */
    double arrival_time;    /* seconds on the server clock; < 0 = now            */
    double deadline;        /* seconds on the server clock by which it must be
                               done; a request still queued or running after it
                               is dropped (ISG_REQ_EXPIRED); <= 0 = none         */
} isg_request;

typedef struct {
    int32_t state;          /* ISG_REQ_QUEUED / RUNNING / DONE                   */
    int64_t sweeps_done;    /* n_sweeps once done                                */
    int64_t B, M, Q;        /* final observables (state DONE)                    */
    double t_arrival, t_admit, t_done;  /* server clock (s); t_done from a CUDA
                               event after the request's last device work        */
    int64_t records;        /* periodic records not yet read                     */
    int32_t error;          /* ISG_REQ_FAILED: the status that failed it (e.g.
                               ISG_ERR_OOM from its allocation); else ISG_OK     */
} isg_result;

isg_status isg_server_create(const isg_server_desc *desc, isg_server **out);
void isg_server_destroy(isg_server *srv);  /* waits for the device; NULL accepted */
/* Queue a request; *id identifies it.  ISG_ERR_OOM if it can never fit. */
isg_status isg_server_submit(isg_server *srv, const isg_request *req, uint64_t *id);
/* One scheduling round (asynchronous device work); counts after it.  A
 * request whose allocation or launch fails is failed alone (ISG_REQ_FAILED,
 * its memory freed); the others go on. */
isg_status isg_server_step(isg_server *srv, int32_t *active, int32_t *queued);
/* Take a queued or running request out of the schedule: it never starts, or
 * stops after the chunk already queued on the device (the call waits for
 * that chunk), and its device memory is freed; state ISG_REQ_CANCELLED.
 * ISG_ERR_INVALID for an unknown request or one that already left the
 * schedule (done, cancelled, expired, failed). */
isg_status isg_server_cancel(isg_server *srv, uint64_t id);
/* Rounds until every submitted request is done (waits for arrivals). */
isg_status isg_server_drain(isg_server *srv);
isg_status isg_server_poll(isg_server *srv, uint64_t id, isg_result *out);
/* Periodic records of a finished, kept request (as isg_read_records; a
 * failed record is passed over and reported as ISG_ERR_DEVICE_TIMEOUT). */
isg_status isg_server_read_records(isg_server *srv, uint64_t id, isg_obs *out, int64_t max,
                                   int64_t *count);
/* Final lattice of a finished, kept request (L*L host bytes).  Synchronises. */
isg_status isg_server_get_lattice(isg_server *srv, uint64_t id, int8_t *out);
/* Free the device memory of a finished request. */
isg_status isg_server_release(isg_server *srv, uint64_t id);
/* Seconds since creation (the clock of arrival and completion times). */
double isg_server_clock(const isg_server *srv);
/* Spin-flip attempts of finished requests; bytes held; budget. */
isg_status isg_server_stats(const isg_server *srv, double *flips_done, size_t *bytes_in_use,
                            size_t *budget);

/* ---------------------------------------------------------------------------
 * Row slabs: the domain decomposition with which the paper runs ONE lattice
 * on many GPUs (Introduction; Table I: L = 2^22 on 64 GPUs).  A slab owns
 * the global rows y0 .. y0 + rows - 1 of an L x L lattice (one slab per
 * process or GPU) and keeps, per colour, one halo row above (global row
 * y0 - 1, periodic) and one below (global row y0 + rows).
 *
 * One sweep t of the whole lattice, on every slab:
 *   1. colour-1 halos: isg_slab_edges(colour 1) -> first / last owned row;
 *      each slab's first row goes to the slab above as its `below` halo and
 *      its last row to the slab below as its `above` halo (periodic, a
 *      single slab is its own neighbour); isg_slab_set_halos(colour 1);
 *   2. isg_slab_half_sweep(colour 0, beta(t));
 *   3. the same exchange for colour 0;
 *   4. isg_slab_half_sweep(colour 1, beta(t)).
 * Random words are keyed by the global site, so the slabs together evolve
 * bit for bit as the lattice created whole with the same seed.  After a
 * sweep the colour-0 halos are current (the colour-1 halos are one
 * half-sweep old), and isg_slab_measure gives the slab's part of every
 * observable: the lattice's B, M and Q are the sums over slabs, its row
 * sums the slabs' row sums in slab order, its column sums the sums of the
 * slabs' column sums.  No call moves data between
 * slabs: the caller does (host memory, peer copies or a collective
 * library), so the library itself stays single-GPU.
 * ------------------------------------------------------------------------- */
typedef struct isg_slab isg_slab;

typedef struct {
    int32_t model;    /* ISG_ISING or ISG_BLUME_CAPEL                           */
    int64_t L;        /* side of the whole lattice (a valid L)                  */
    int64_t y0;       /* first owned global row: a multiple of 16               */
    int64_t rows;     /* owned rows: a multiple of 16, >= 16, y0 + rows <= L    */
    uint64_t seed;    /* Philox key of the whole lattice                        */
    double delta;     /* Blume-Capel crystal field                              */
    void *stream;     /* cudaStream_t for all work, NULL = default stream       */
} isg_slab_desc;

/* Bytes of one edge or halo row of one colour: L/16 (Ising) or L/8
 * (Blume-Capel: the occupancy words, then the sign words), in the plane
 * layout of isg_save.  0 if the model or L is invalid. */
size_t isg_slab_edge_bytes(int32_t model, int64_t L);

/* Allocate the slab's planes ((rows + 2) rows per colour plane) on the
 * current device; spins undefined, halos zero.  *out NULL on failure. */
isg_status isg_slab_create(const isg_slab_desc *desc, isg_slab **out);
/* Free everything (waits for the stream).  NULL accepted. */
void isg_slab_destroy(isg_slab *slab);
/* Hot start of the owned rows, equal to those rows of the whole lattice's
 * isg_lattice_init_random; sweep counter 0. */
isg_status isg_slab_init_random(isg_slab *slab);
/* Owned rows from / to rows*L host bytes s[(y - y0) L + x]; set also sets the
 * sweep counter to t.  ISG_ERR_INVALID on a value outside the model's set.
 * Synchronise. */
isg_status isg_slab_set(isg_slab *slab, const int8_t *host, int64_t t);
isg_status isg_slab_get(isg_slab *slab, int8_t *out);
/* Copy colour `colour`'s first and last owned rows (isg_slab_edge_bytes
 * each) to caller memory, host or device (any pointer the CUDA runtime can
 * address).  Queued on the stream; waits for it when a destination is host
 * memory. */
isg_status isg_slab_edges(isg_slab *slab, int32_t colour, void *first, void *last);
/* Load colour `colour`'s halo rows: `above` = global row y0 - 1 (the last
 * row of the slab above), `below` = global row y0 + rows (the first row of
 * the slab below).  Host or device memory; waits for the stream when a
 * source is host memory. */
isg_status isg_slab_set_halos(isg_slab *slab, int32_t colour, const void *above,
                              const void *below);
/* Half-sweep of colour `colour` of the owned rows at the slab's sweep
 * counter t with inverse temperature beta (reads the other colour's halos).
 * Colour 1 completes the sweep and advances the counter.  Asynchronous. */
isg_status isg_slab_half_sweep(isg_slab *slab, int32_t colour, double beta);
/* The slab's observables: B over the four bonds of every owned colour-1
 * site (every bond joins a colour-0 and a colour-1 site, so the slabs' B
 * add up to the lattice's; reads the colour-0 halos, current after a
 * sweep), M, Q, row_sums[0..rows) of the owned rows and col_sums[0..L) of
 * the owned part of each column, into caller HOST arrays (either may be
 * NULL); out->sweep = the sweep counter.  Synchronises. */
isg_status isg_slab_measure(isg_slab *slab, isg_obs *out);
/* Sweep counter, L, y0, rows, model. */
isg_status isg_slab_info(const isg_slab *slab, int64_t *sweep, int64_t *L, int64_t *y0,
                         int64_t *rows, int32_t *model);

/* Correlation function along the axes (Eq. (2)) of the current lattice: for
 * each distance r[k] (0 <= r[k] < L) the exact sums
 *   out_x[k] = sum_{x,y} s(x,y) s(x + r[k], y),
 *   out_y[k] = sum_{x,y} s(x,y) s(x, y + r[k])   (periodic),
 * so that C(r) = (out_x + out_y) / (2 L^2) averages the two axes and the
 * energy of Eq. (3) is (out_x + out_y at r = 1) / L^2 up to its sign.  One
 * pass over the lattice per distance.  Synchronises. */
isg_status isg_correlation(isg_lattice *lat, int64_t nr, const int64_t *r, int64_t *out_x,
                           int64_t *out_y);

/* Integral coherence length xi = I2 / I1 (Appendix C), I_n = int_0^{r_cut}
 * r^n C(r) dr by the trapezoid rule over the n sampled points r[0] < r[1] <
 * ... (host FP64; points beyond r_cut ignored).  NaN if I1 <= 0 or n < 2.
 * The paper's choice of r_cut from the errors of C, and its fitted tail
 * F(r), are analysis steps left to the caller. */
double isg_xi_integral(int64_t n, const double *r, const double *c, double r_cut);

/* Swendsen-Wang iteration of the s = +-1 spins (Appendix B: the Blume-Capel
 * equilibrium runs alternate Metropolis sweeps, which change s^2, with
 * Swendsen-Wang cluster updates restricted to s = +-1; for Ising every site
 * takes part).  Bond (i, j), j the +x (d = 0) or +y (d = 1) neighbour of
 * site i = y L + x, is active iff s_i = s_j != 0 and u < rne(2^32 (1 -
 * e^{-2 beta})), u the word i & 3 of Philox4x32-10 with key (lo, hi) of
 * the lattice seed and counter (lo(i >> 2), hi(i >> 2), k, 4 + d), k the
 * value of isg_sw_iterations before the call.  A cluster (connected
 * component of active bonds) flips s -> -s iff the word r & 3 of counter
 * (lo(r >> 2), hi(r >> 2), k, 6) is >= 2^31, r its smallest site index.
 * Sites with s = 0 never bond nor flip.  The sweep counter is unchanged.
 * Needs L <= ISG_SW_MAX_L; allocates L^2 4-byte labels on first use (kept
 * until destroy).  Errors: INVALID (beta < 0 or not finite, L too large,
 * 2^32 iterations), OOM, DEVICE_TIMEOUT (a bounded device loop ran out;
 * not expected).  Synchronises. */
#define ISG_SW_MAX_L 32768
isg_status isg_swendsen_wang(isg_lattice *lat, double beta);

/* Cluster labels of the last Swendsen-Wang iteration (before its flips):
 * out[y*L + x] = smallest site index of the site's cluster (its own index
 * for s = 0).  out: L*L host int32.  INVALID if no iteration has run.
 * Synchronises. */
isg_status isg_sw_labels(isg_lattice *lat, int32_t *out);

/* Swendsen-Wang iterations done on this lattice (reset by the init calls,
 * kept by isg_save / isg_load). */
isg_status isg_sw_iterations(const isg_lattice *lat, int64_t *count);

/* Fault injection, for testing callers' and the library's error paths on
 * the host (no device fault is ever raised).  what = ISG_INJECT_ALLOC: the
 * `after`-th device allocation the library makes from now on (counting this
 * process's calls of every object) fails as out of memory -- nothing is
 * allocated and the call reports ISG_ERR_OOM after freeing what it had
 * allocated.  what = ISG_INJECT_LAUNCH: the `after`-th sweep kernel launch
 * (single-lattice, slab, multi-lattice or persistent ensemble / server
 * launch) is skipped and the call reports ISG_ERR_CUDA.  what =
 * ISG_INJECT_WAIT: the `after`-th record pass that streams its rows through
 * shared memory (lattices with L a multiple of 16384) announces 16 bytes more
 * than it copies in one block, so that block's bounded waits run out (about
 * 4 s); the pass marks the record failed and the call that reads it (or
 * isg_read_records, which drops it) reports ISG_ERR_DEVICE_TIMEOUT.  Each
 * injection fires once; after = 0 disarms it.  Process-wide, thread-safe. */
#define ISG_INJECT_ALLOC 1
#define ISG_INJECT_LAUNCH 2
#define ISG_INJECT_WAIT 3
isg_status isg_debug_inject(int32_t what, int64_t after);

/* Energy per spin (-B + Delta Q) / L^2 of one record. */
double isg_energy_density(const isg_obs *obs, int64_t L, double delta);

/* Human-readable message about the last failure in the calling thread. */
const char *isg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ISG_H */
