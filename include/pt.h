/*
 * pt.h -- C ABI of libpt: Metropolis-Hastings with Parallel Tempering for the periodic
 * two-dimensional Ising model on one NVIDIA B300 (sm_103a).
 *
 * Method (arXiv 2512.03825):
 *   - Sec. 2.2, Eq. 3: E(sigma) = h * sum_i sigma_i - J * sum_<ij> sigma_i sigma_j on an L x L
 *     periodic square lattice, every nearest-neighbour bond counted once. The field enters
 *     with the paper's + sign, so h > 0 favours negative magnetisation.
 *   - Sec. 2.2, Eq. 2: Boltzmann target P(E) ~ exp(-beta E), k_B = 1, beta = 1/T.
 *   - Sec. 2.1, Eq. 1: Metropolis acceptance min(1, exp(-beta dE)) for single-spin flips.
 *   - Sec. 3: R replicas at R temperatures run in intervals; between intervals neighbouring
 *     temperatures exchange states, pairs (0,1),(2,3),... on the first swap iteration and
 *     (1,2),(3,4),... on the next, alternating, with probability
 *     e^x / (1 + e^x), x = (beta_k - beta_k+1)(E_k - E_k+1).
 *
 * Exact integer form (all decisions are bit-reproducible):
 *   - J and h are quantised: s = smallest integer in 1..1000 with s*J and s*h within 1e-9
 *     of integers; J_int = round(s*J), h_int = round(s*h), |J_int|, |h_int| <= 2^20.
 *     E_int = s * E is an exact int64.
 *   - Sweep t (t = 0, 1, ... counted since pt_create) visits colour 0 of the checkerboard
 *     ((x + y) even) and then colour 1. The replica in slot r at site i = y*L + x draws
 *     u = Philox4x32-10(key = seed, ctr = {i, lo32(t), r >> 2, 0 | hi32(t) << 8}) word r & 3
 *     and flips when dE_int <= 0 or u < floor(2^32 * exp(-(beta * dE_int) / s)), where
 *     dE_int = 2 sigma (J_int * sum_nb sigma_nb - h_int) and beta is the inverse temperature
 *     the slot currently runs at (all in IEEE double, libm exp, no fused operations).
 *   - Replica slot r starts at temperature index r with spins sigma = +1 iff bit 31 of
 *     Philox(ctr = {i, 0, r >> 2, 2}) word r & 3 is set.
 *   - After every sweep that leaves the total sweep count a multiple of exchange_every (> 0),
 *     swap iteration e (e = 0, 1, ... since pt_create) tries the pairs (k, k+1), k = e & 1,
 *     e & 1 + 2, ...: with n = E_int(at k) - E_int(at k+1), y = ((beta_k+1 - beta_k) * n) / s
 *     and u = Philox(ctr = {k, lo32(e), 0, 1 | hi32(e) << 8}) word 0, the pair swaps when
 *     u < S with S = 0 for y > 44, S = 2^32 for y < -44 and floor(2^32 / (1 + exp(y)))
 *     otherwise. A swap exchanges the two slots' temperature indices; configurations never
 *     move in memory.
 *
 * Conventions for every call:
 *   - Return value 0 (PT_OK) on success, a negative PT_E* code otherwise; pt_strerror() turns
 *     a code into text and pt_last_error() gives the detail of the last failure on the
 *     calling thread.
 *   - A problem whose device work failed is poisoned: later calls on it return PT_ESTATE
 *     until it is destroyed.
 *   - Output arrays are owned by the caller and must hold the stated number of elements;
 *     every array argument is host memory unless stated otherwise.
 *   - One pt_problem must not be used from two host threads at once.
 *   - pt_sweep and pt_sweep_batch are asynchronous on the problem's CUDA stream; every
 *     getter synchronises that stream before it returns.
 *   - The library needs a CUDA device of compute capability 10.3 (B300). Without one every
 *     call that touches the device returns PT_ENODEV; nothing falls back to the CPU.
 */
#ifndef PT_H_
#define PT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PT_OK 0
#define PT_EINVAL (-1)   /* malformed argument */
#define PT_ENOMEM (-2)   /* device or host allocation failed */
#define PT_ECUDA (-3)    /* a CUDA call failed */
#define PT_ETIMEOUT (-4) /* a device-side wait gave up */
#define PT_ESTATE (-5)   /* the problem was poisoned by an earlier failure */
#define PT_ENODEV (-6)   /* no usable sm_103 device */
#define PT_EINTERNAL (-7)

#define PT_MAX_L 16384
#define PT_MAX_R 2048

typedef struct pt_problem pt_problem; /* opaque; owned by the library until pt_destroy */

/* Create one PT problem (Sec. 3, initialisation phase): L x L periodic lattice (L even,
 * 4 <= L <= PT_MAX_L), R temperatures with inverse temperatures betas[0..R-1] (finite,
 * >= 0; copied; their order defines the temperature index; 1 <= R <= PT_MAX_R), coupling J,
 * field h, 64-bit seed. Allocates the device state (about L*L*ceil(R/32)*4 bytes of spins
 * plus the threshold tables) through the allocator of pt_set_allocator (cudaMalloc by
 * default), draws the initial spins on the device, and stores the handle in *out. The
 * problem runs on the legacy default stream until pt_set_stream. Errors: PT_EINVAL,
 * PT_ENOMEM, PT_ECUDA, PT_ENODEV. */
int pt_create(int L, const double* betas, int R, double J, double h, uint64_t seed,
              pt_problem** out);

/* Options of pt_create_ex. `size` is sizeof(pt_options) as the caller was compiled (fields
 * past it keep their defaults), so later versions can add fields.
 *   swap_rule  PT_SWAP_BARKER (default; the paper's rule, Sec. 3): accept with probability
 *              e^x / (1 + e^x) = 1 / (1 + e^y), S(y) = floor(2^32 / (1 + exp(y))), 0 above
 *              y = 44 and 2^32 below -44;
 *              PT_SWAP_METROPOLIS (an option the paper does not use): accept with
 *              probability min(1, e^x) = min(1, e^-y), S(y) = 2^32 for y <= 0, 0 above
 *              y = 44, floor(2^32 * exp(-y)) in between.
 *   (x, y, n and s as in the swap rule at the top of this file.) Both rules satisfy detailed
 *   balance for the pair, p(y) / p(-y) = e^-y.
 *   stream     the problem's stream from the start (a cudaStream_t, as pt_set_stream).
 *              NULL (default): the legacy default stream, and pt_create_ex returns once the
 *              problem is initialised. Otherwise the initialisation (one host-to-device copy
 *              of thresholds and tables, the initial spins, the plane thresholds) is queued
 *              on that stream and pt_create_ex returns without waiting; a device failure
 *              during it is reported, and poisons the problem, at the next call that
 *              synchronises. */
#define PT_SWAP_BARKER 0
#define PT_SWAP_METROPOLIS 1
typedef struct pt_options {
  uint32_t size;
  int32_t swap_rule;
  void* stream;
} pt_options;

/* pt_create with options (NULL: the defaults of pt_create). PT_EINVAL for an unknown swap
 * rule or a size outside 4..4096. The thresholds and tables that a problem's creation copies
 * to the device depend only on its ladder, J, h, swap rule and (for small lattices) L, not
 * on the seed: up to 64 MiB of them per problem are kept in page-locked host memory after
 * the first creation (at most 1 GiB in all) and copied from there by later creations with
 * the same parameters. */
int pt_create_ex(int L, const double* betas, int R, double J, double h, uint64_t seed,
                 const pt_options* opt, pt_problem** out);

/* Release the problem and its device memory (synchronises its stream first). NULL is a
 * no-op. */
void pt_destroy(pt_problem* p);

/* Run the problem's future work on `cuda_stream` (a cudaStream_t, e.g. a torch stream
 * handle). Synchronises the previous stream first. */
int pt_set_stream(pt_problem* p, void* cuda_stream);

/* Sec. 3, execution phase: n >= 0 sweeps, with a swap iteration after every sweep that
 * leaves the total sweep count a multiple of exchange_every (0 = no swaps; < 0 is
 * PT_EINVAL). pt_sweep(a, m) followed by pt_sweep(b, m) equals pt_sweep(a + b, m).
 * Launches the problem's kernels (the plain path: see pt_set_sweep_tuning) and returns
 * without waiting. */
int pt_sweep(pt_problem* p, int64_t n, int exchange_every);

/* How pt_sweep runs this problem (results never depend on it):
 *   PT_SWEEP_AUTO       -- persistent when the problem fits, else launches (the default);
 *   PT_SWEEP_LAUNCHES   -- one launch per half sweep, plus an energy-count and an exchange
 *                          launch after each sweep that ends with a swap iteration;
 *   PT_SWEEP_PERSISTENT -- one cooperative launch per call (up to 65536 sweeps each) whose
 *                          CTAs meet at grid barriers between half sweeps and all compute
 *                          the swap iterations themselves. It fits when every 32-replica
 *                          plane gets at least one CTA of one resident wave and no thread
 *                          owns more than 255 words of a colour; pt_sweep returns PT_EINVAL
 *                          otherwise.
 *   PT_SWEEP_BANDS      -- the persistent kernel with each CTA owning a band of whole rows
 *                          of a plane, kept in shared memory with one halo row on either
 *                          side: colour 0 is updated on the band and again, from the same
 *                          inputs, on its two halo rows, so colour 1 needs no grid barrier
 *                          before it and a sweep takes one grid barrier instead of two (for
 *                          small lattices, where the barriers dominate). It fits when the
 *                          persistent kernel fits with at least two bands per plane and a
 *                          band's copies fit 48 KB of shared memory; pt_sweep returns
 *                          PT_EINVAL otherwise. PT_SWEEP_PERSISTENT never uses the bands;
 *                          PT_SWEEP_AUTO uses them where they measured faster.
 * words_per_thread (1..255, 0 = the default 1) sets how many words of each colour a thread
 * of the persistent kernel aims to own: the CTA count is the one that gives that many,
 * capped at one resident wave. PT_EINVAL for an unknown strategy or a count out of range. */
#define PT_SWEEP_AUTO 0
#define PT_SWEEP_LAUNCHES 1
#define PT_SWEEP_PERSISTENT 2
#define PT_SWEEP_BANDS 3
int pt_set_sweep_tuning(pt_problem* p, int strategy, int words_per_thread);

/* The problem's sweep strategy, words-per-thread setting and the CTA count the persistent
 * kernel would use (0 when the problem does not fit it). Any pointer may be NULL. */
int pt_get_sweep_tuning(pt_problem* p, int* strategy, int* words_per_thread, int* grid);

/* Time limit of each wait of the persistent kernel at a grid barrier, in seconds
 * (0 < seconds <= 60; default 1). A wait that runs out stores PT_ETIMEOUT in the problem's
 * device status, every CTA leaves the kernel, and the next pt_synchronize (or getter)
 * returns PT_ETIMEOUT and poisons the problem; the CUDA context stays usable. */
int pt_set_wait_limit(pt_problem* p, double seconds);

/* Test support for the bounded wait; the paper has no counterpart. The next persistent launch
 * of this problem waits at its first grid barrier for `arrivals` (>= 0) more CTAs than it
 * has (in a PT_BATCH_FLOW batch: its first colour-1 wait expects that many more tiles), so
 * that the wait runs out after the wait limit and the launch ends with PT_ETIMEOUT as
 * described above. Applies to one launch. */
int pt_debug_stall_barrier(pt_problem* p, int arrivals);

/* The debug build of the library (libpt_debug.so, compiled with PT_DEBUG) stands in for a
 * memory and race checker on small cases; the paper has no counterpart. In it every
 * spin-word index a kernel reads or writes is checked against the word range of its plane and
 * colour before the access, and so is every count-buffer index and trace row; every store of
 * a half sweep tags its word with the number of that half sweep, so a word stored twice in
 * one half sweep (two threads owning one site) is caught. A failed check never traps: it is
 * recorded, the access is redirected to the start of its array or skipped, and the
 * problem's status makes its next synchronising call return PT_EINTERNAL. The release library
 * compiles none of these checks; its kernels are unchanged by them.
 *
 * pt_debug_build: 1 in the debug build, 0 in the release library. */
int pt_debug_build(void);

/* The problem's record of failed checks (debug build): how many (*violations), the kind of
 * the first (*first_kind: 1 a spin-word load, 2 a spin-word store outside its plane and
 * colour, 3 a spin word stored twice in one half sweep, 4 a count-buffer index, 5 a trace
 * row, 6 a single-flip word outside its plane; 0 none) and the index it was given; and
 * *unwritten, the spin words that the problem's last sweep did not store in their own half
 * sweep (0 when no sweep has run since pt_create or pt_load). Any pointer may be NULL.
 * Synchronises the stream and does not poison the problem. PT_EINVAL in the release
 * library. */
int pt_debug_report(pt_problem* p, uint64_t* violations, int32_t* first_kind,
                    uint64_t* first_index, uint64_t* unwritten);

/* Test support of the debug build: the next launch of the one-launch-per-half-sweep kernel
 * (PT_SWEEP_LAUNCHES) of this problem plants one mistake in its first thread, which the
 * checks must catch: kind 1 stores that thread's first word a second time, unchanged (a double
 * write), kind 2 asks for a neighbour word one past its colour's range (the check redirects
 * the load into the range). 0 clears. PT_EINVAL in the release library or for another kind. */
int pt_debug_inject(pt_problem* p, int kind);

/* The single-spin-flip variant: the paper's "iteration" (Sec. 2.1, the MH step whose trial
 * state flips one spin) read as one Metropolis trial at one uniformly chosen site of every
 * replica. n >= 0 iterations of every replica; after every iteration that leaves the
 * iteration count (since pt_create) a multiple of exchange_every (> 0; 0 = none), one swap
 * iteration exactly as after sweeps, sharing their swap index e. Iteration i of the replica
 * in slot r draws u = Philox4x32-10(key = seed, ctr = {lo32(i), r, 0, 3 | hi32(i) << 8}):
 * the site is floor(u.word0 * L^2 / 2^32) (i = y*L + x) and the trial, with dE_int and the
 * threshold T of a sweep's trial, flips when u.word1 < T. One cooperative launch per call
 * (one thread per replica; waits bounded as for PT_SWEEP_PERSISTENT); trace rows are not
 * written. Asynchronous like pt_sweep. */
int pt_flip(pt_problem* p, int64_t n, int exchange_every);

/* How pt_flip runs (results never depend on it): shared_memory != 0 (the default) keeps the
 * replicas of a block in shared memory as private bit arrays when k >= 1 of them (a power of
 * two) fit one CTA and the blocks one resident wave, else the kernel reads and flips the
 * shared spin words in global memory (atomic XOR per flip). */
int pt_set_flip_tuning(pt_problem* p, int shared_memory);

/* Single-spin-flip iterations done since pt_create. */
int pt_iterations(pt_problem* p, uint64_t* iterations_done);

/* Advance `count` problems together (Sec. 3's execution phase for many independent
 * problems): problem j runs n[j] >= 0 sweeps with exchange_every[j] (same meaning as
 * pt_sweep). The batched strategy is pt_set_batch_tuning's: by default one launch per half
 * sweep over warp tiles of every problem plus one exchange launch per sweep that ends with a
 * swap iteration (PT_BATCH_FLAT, or PT_BATCH_QUEUE), in the parts of pt_set_batch_streams;
 * PT_BATCH_FLOW and PT_BATCH_CLUSTER make one persistent launch per call. All problems must be on the same stream and device,
 * none listed twice. Results are bit-identical to calling pt_sweep on each problem alone.
 * count = 0 does nothing and returns PT_OK; count < 0, or missing arrays, PT_EINVAL. */
int pt_sweep_batch(pt_problem* const* problems, int count, const int64_t* n,
                   const int* exchange_every);

/* pt_sweep_batch without any allocation. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory while they run -- code inside a
 * memory budget it has already fixed, code whose device memory belongs to an allocator this
 * library cannot see, or code that must not let an allocation synchronise the device or fail
 * part-way. It runs the lock-step kernels of pt_sweep_batch (bit-identical results), handing
 * the tiles out as PT_BATCH_QUEUE does when that strategy is set (pt_set_batch_tuning) and
 * as PT_BATCH_FLAT does under any other strategy, but keeps the per-call work lists
 * (problem descriptors, work tiles, per-warp tile offsets) in one 1 MiB array of device
 * memory that the library defines at file scope; every GPU that loads the library holds
 * that array until the process exits. The work lists of a batch take about 256 bytes per
 * problem plus 16 bytes per 512-word tile of every 32-replica plane plus 4 bytes per
 * resident warp; a batch that does not fit (or lists more than 2048 problems, or needs more
 * than 65536 tiles) is rejected with PT_EINVAL and a message saying so, before anything is
 * launched. No call allocates: not on the device (no cudaMalloc, cudaMallocAsync or
 * cudaFree) and not on the host heap; the host side builds the lists in fixed arrays.
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current. Every call shares the one array and overwrites what the
 * previous call left there (nothing in it has to start at zero: each call writes every part
 * it reads). Calls are serialised on the host and each call waits until its lists have been
 * copied to the device, but two calls whose kernels overlap on the GPU (different streams,
 * different problems) race on the array: issue them on one stream, or synchronise between
 * them. The call cannot be recorded into a CUDA graph (its copies read host arrays that the
 * next call overwrites, and it waits for them): while the problems' stream is being
 * captured it returns PT_EINVAL before queuing anything, and the problems stay usable. */
int pt_sweep_batch_static(pt_problem* const* problems, int count, const int64_t* n,
                          const int* exchange_every);

/* How pt_sweep_batch runs (chosen by the autotuner; results never depend on it):
 *   PT_BATCH_FLAT    -- all problems advance sweep by sweep together; every half sweep is
 *                       one launch over equal-sized word tiles of all problems, followed by
 *                       an exchange launch when any problem is due; the host deals the
 *                       tiles to the warps (longest processing time first);
 *   PT_BATCH_QUEUE   -- PT_BATCH_FLAT with the tiles handed out on the device: one tile per
 *                       warp first, then each warp that finishes a tile takes the next
 *                       (largest first) from a counter, so the warps finish together
 *                       however the SMs' loads differ; the tiles of the cheapest quarter of
 *                       the work are cut in two, so each launch ends on small tiles;
 *   PT_BATCH_CLUSTER -- one persistent kernel; a problem with L >= joint_min_L runs on a
 *                       whole thread-block cluster of `cluster` CTAs (1 to 16) for all of its
 *                       sweeps, smaller ones on a single CTA;
 *   PT_BATCH_FLOW    -- the tiles of PT_BATCH_FLAT in one cooperative launch per call (one
 *                       per mode: J, h with h = 0 and J > 0, and the rest), whose warps run
 *                       all sweeps and order each problem's half sweeps and swap iterations
 *                       by per-problem counters instead of launches. Each wait is bounded by
 *                       the problem's wait limit (pt_set_wait_limit); a wait that runs out
 *                       marks every problem of the call PT_ETIMEOUT, reported by the next
 *                       pt_synchronize or getter. pt_debug_stall_barrier applies to it too.
 * pt_sweep_batch_static hands its tiles out as PT_BATCH_QUEUE does when that strategy is
 * set, and as PT_BATCH_FLAT does otherwise. A batch with a traced problem runs
 * PT_BATCH_QUEUE when it is set, and PT_BATCH_FLAT otherwise. Applies to later batches of
 * every problem. PT_EINVAL for an unknown strategy, cluster outside 1..16 or
 * joint_min_L < 4. */
#define PT_BATCH_FLAT 0
#define PT_BATCH_CLUSTER 1
#define PT_BATCH_FLOW 2
#define PT_BATCH_QUEUE 3
int pt_set_batch_tuning(int strategy, int cluster, int joint_min_L);
int pt_get_batch_tuning(int* strategy, int* cluster, int* joint_min_L);

/* Tile size of PT_BATCH_FLAT, PT_BATCH_QUEUE, PT_BATCH_FLOW and pt_sweep_batch_static:
 * each problem's words of one colour and plane are cut into max(1, round(words /
 * tile_words)) equal tiles, one warp's unit of work (tile_words / 32 words per lane;
 * default 512). Smaller tiles balance the warps better and cost more per-tile setup;
 * results never depend on it. tile_words: a multiple of 32 in [PT_TILE_WORDS_MIN,
 * PT_TILE_WORDS_MAX], else PT_EINVAL. Applies to later batches of every problem. */
#define PT_TILE_WORDS_MIN 64
#define PT_TILE_WORDS_MAX 1024
int pt_set_batch_tile_words(int tile_words);
int pt_get_batch_tile_words(int* tile_words);

/* Streams of PT_BATCH_FLAT and PT_BATCH_QUEUE (1..PT_BATCH_STREAMS_MAX, default 1; set by the
 * autotuner): pt_sweep_batch splits the batch into that many parts of about equal work (L*L
 * times planes times sweeps, heaviest problem first onto the lightest part) and advances each
 * part on its own CUDA stream -- the first on the problems' stream, the others on side streams
 * that the library owns per device, which wait for everything queued on the problems' stream
 * before the call and which the problems' stream waits for at its end, so the call is ordered
 * on the problems' stream as before. Sweep j of one part runs beside sweep j of the others:
 * one part's exchange launch, launch gaps and last tiles overlap the others' half sweeps.
 * Results never depend on it. Calls that use the side streams are serialised on the host per
 * device. pt_sweep_batch_static always runs one part. PT_EINVAL outside the range. Applies to
 * later batches of every problem. */
#define PT_BATCH_STREAMS_MAX 4
int pt_set_batch_streams(int streams);
int pt_get_batch_streams(int* streams);

/* Graph replay of PT_BATCH_FLAT and PT_BATCH_QUEUE batches (0 = off, the default; 1 = on; set
 * by the autotuner): the launches of a batch call depend only on its shape -- per problem, in
 * call order, L, R, the mode, n, exchange_every, the phase of its exchange schedule and
 * whether a trace is on -- and on the tile size, schedule, streams and stream. With replay on,
 * the first call of a shape builds its work lists in device memory of their own and captures
 * its launches into a CUDA graph; a later call of the same shape copies the problems'
 * descriptors (counters and device arrays) and launches that graph: one launch instead of
 * about three per part and sweep, which frees the host on long calls and on batches of small
 * problems, where issuing the launches can take longer than running them. The first call of
 * a shape is slower (lists built in blocking copies, capture, instantiation); the library
 * keeps four shapes per device (least recently used dropped; dropping one waits for the
 * device). A call on the legacy default stream, or made while the problems' stream is being
 * captured, launches as without replay. Results never depend on it. PT_EINVAL for other
 * values. */
int pt_set_batch_graphs(int on);
int pt_get_batch_graphs(int* on);

/* Energies E = E_int / s of the configurations at each temperature index, out[R]. */
int pt_energies(pt_problem* p, double* out);

/* Magnetisations M = sum_i sigma_i at each temperature index, out[R]. */
int pt_magnetisations(pt_problem* p, double* out);

/* Swap statistics per temperature pair (k, k+1): attempts and acceptances, each [R-1]
 * (either pointer may be NULL; nothing is written when R == 1). */
int pt_swap_stats(pt_problem* p, uint64_t* attempted, uint64_t* accepted);

/* Exact integer observables per temperature index: E_int[R], M[R] (either may be NULL) and
 * the quantisation scale s (may be NULL). */
int pt_energies_int(pt_problem* p, int64_t* E_int, int64_t* M, int64_t* scale);

/* Spins (+1 / -1, row-major [L][L], site (x, y) at y*L + x) of the configuration at
 * temperature index k. */
int pt_get_spins(pt_problem* p, int k, int8_t* out);

/* Overwrite the configuration at temperature index k with in[L*L] (values +1 / -1 only,
 * else PT_EINVAL). */
int pt_set_spins(pt_problem* p, int k, const int8_t* in);

/* slot_of_temp[R]: the replica slot (chain) currently at each temperature index (Sec. 3:
 * a swap exchanges the temperatures of two slots, so this map is the result of every swap
 * so far). Synchronises the problem's stream. PT_EINVAL for a NULL output. */
int pt_chain_map(pt_problem* p, int32_t* slot_of_temp);

/* The same map under the name of the exchange step's permutation: identical to
 * pt_chain_map. */
int pt_temperature_map(pt_problem* p, int32_t* slot_of_temp);

/* Sweeps and swap iterations done since pt_create (either pointer may be NULL). */
int pt_counters(pt_problem* p, uint64_t* sweeps_done, uint64_t* exchanges_done);

/* The results of `count` problems in one transfer. For problem j: E_int[j] and M[j] (R_j
 * values each, by temperature index, as pt_energies_int), slot_of_temp[j] (R_j, as
 * pt_chain_map), attempted[j] and accepted[j] (R_j - 1 values, as pt_swap_stats; nothing for
 * R_j = 1). Any of the five pointer arrays may be NULL, and so may any entry of one; the
 * caller owns every array. The problems must share a stream and a device (as in
 * pt_sweep_batch). Recomputes the energies from the current spins like the single getters
 * (one count launch over the words of every problem), packs every problem's record with one
 * kernel into a stream-ordered scratch buffer and copies it back once: one synchronisation
 * instead of several per problem and getter. A problem listed more than once is read once
 * and its record given to each of its entries. A
 * problem whose device work reported a status (PT_ETIMEOUT, ...) is poisoned as by
 * pt_synchronize and its arrays are left untouched; the call returns the first such error
 * after filling the others. PT_EINVAL for count < 0, a NULL or repeated-on-another-stream
 * problem; PT_ENOMEM if the scratch buffer cannot be had. */
int pt_read_batch(pt_problem* const* problems, int count, int64_t* const* E_int,
                  int64_t* const* M, int32_t* const* slot_of_temp, uint64_t* const* attempted,
                  uint64_t* const* accepted);

/* Checkpoints. pt_save writes the problem's whole sampler state into buf (host memory of
 * at least pt_checkpoint_bytes(p) bytes; synchronises the stream); pt_load creates a new
 * problem (on the current device, through the current allocator) that continues exactly as
 * the saved one would have: same spins, temperature map, sweep and swap counters, swap
 * statistics, single-flip iterations, seed, couplings and swap rule. A trace ring is not part
 * of the state. The
 * bytes, little-endian, no padding:
 *   0   "PTCKPT02"          8 bytes
 *   8   L, R                uint32 each
 *   16  J, h                double each
 *   32  seed, t, e          uint64 each (sweeps and swap iterations done)
 *   56  swap rule, 0        int32 each
 *   64  it                  uint64 (single-spin-flip iterations done)
 *   72  betas[R]            double
 *       slot_of_temp[R]     int32 (a permutation)
 *       attempted[R-1], accepted[R-1]   uint64
 *       spins               uint32 [W][2][L][L/2], W = ceil(R/32): slot r is bit r % 32 of
 *                           plane r / 32, bit set = +1, site (x, y) with colour c = (x+y) & 1
 *                           in word ((w*2 + c)*L + y)*L/2 + x/2; bits of unused slots are 0
 *       FNV-1a 64 of all bytes before it
 * pt_load checks the size, magic, checksum and contents (PT_EINVAL) before it touches a
 * device. */
size_t pt_checkpoint_bytes(const pt_problem* p);
int pt_save(pt_problem* p, void* buf, size_t bytes);
int pt_load(const void* buf, size_t bytes, pt_problem** out);

/* Observable traces: the per-sweep chain of energies and magnetisations at every
 * temperature (the "stored chains" of the paper's CPU programs, Sec. 5), kept on the device in a ring
 * of bounded size. After pt_trace_start(p, capacity) (1 <= capacity <= 2^32 rows), every sweep
 * of pt_sweep or pt_sweep_batch appends one row E_int[R], M[R] by temperature index, taken
 * after the sweep and its swap iteration (if any); the oldest rows are overwritten once
 * `capacity` rows exist. The ring holds capacity * R * 16 bytes of device memory, allocated
 * like the problem's own; restarting replaces the ring. Tracing makes every sweep count the
 * bonds and up spins (a few per cent of a sweep); a batch with a traced problem runs the
 * PT_BATCH_FLAT strategy. pt_trace_stop frees the ring (a no-op without one). Errors:
 * PT_EINVAL, PT_ENOMEM, PT_ECUDA. */
int pt_trace_start(pt_problem* p, int64_t capacity);
int pt_trace_stop(pt_problem* p);

/* Copy up to max_rows of the newest trace rows, oldest first, to E_int[rows][R] and
 * M[rows][R] (either may be NULL); *rows = rows copied (min(max_rows, capacity, sweeps since
 * pt_trace_start)) and *first_sweep = the sweeps done since pt_create when the first of them
 * was taken (either may be NULL). Synchronises the stream. PT_ESTATE without a trace. */
int pt_trace_read(pt_problem* p, int64_t max_rows, int64_t* E_int, int64_t* M,
                  uint64_t* first_sweep, int64_t* rows);

/* Wait for the problem's queued work; reports device-side failures. */
int pt_synchronize(pt_problem* p);

/* Device bytes held by the problem (spins, tables and bookkeeping). */
size_t pt_device_bytes(const pt_problem* p);

/* Device bytes pt_create would allocate for these arguments (0 if they are invalid). Used
 * for admission against a memory budget before creating. */
size_t pt_estimate_device_bytes(int L, const double* betas, int R, double J, double h);

/* Page-locked host memory that the creation-image cache may hold (default 1 GiB). A
 * creation copies its problem's thresholds and tables from an image; images of at most
 * min(64 MiB, limit) bytes are built once into page-locked memory and kept, larger ones are
 * built per creation in pageable memory (0: every image). When the cache would exceed the
 * limit it is emptied; an image that a live problem was created from stays allocated until
 * that problem is destroyed. Always PT_OK. */
int pt_set_image_cache_limit(size_t bytes);

/* Page-locked bytes the creation-image cache holds now. */
size_t pt_image_cache_bytes(void);

/* Route device allocations of later pt_create calls through alloc/free (e.g. the PyTorch
 * caching allocator). alloc(bytes, stream, ctx) returns a device pointer aligned to 256
 * bytes or NULL; free(ptr, stream, ctx) releases it. Pass NULLs to restore cudaMalloc. */
typedef void* (*pt_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*pt_free_fn)(void* ptr, void* stream, void* ctx);
int pt_set_allocator(pt_alloc_fn alloc, pt_free_fn free, void* ctx);

/* Text for a PT_E* code (static storage). */
const char* pt_strerror(int code);

/* Detail of the last failure on the calling thread (static thread-local storage). */
const char* pt_last_error(void);

/* ---- host-side tables, exposed so they can be checked without a GPU ------------------ */

/* The quantisation above: *s, *J_int, *h_int. PT_EINVAL if J or h cannot be quantised. */
int pt_quantise(double J, double h, int64_t* s, int64_t* J_int, int64_t* h_int);

/* Metropolis threshold floor(2^32 * exp(-(beta * dE_int) / s)) for dE_int > 0, 2^32 for
 * dE_int <= 0 (Eq. 1 with Eq. 2). */
uint64_t pt_spin_threshold(double beta, int64_t dE_int, int64_t s);

/* Exchange threshold S of the swap rule above, in [0, 2^32], for the pair with inverse
 * temperatures beta_lo (index k) and beta_hi (index k+1) and energy difference n. Computed
 * from the table the device uses. */
uint64_t pt_swap_threshold(double beta_lo, double beta_hi, int64_t n, int64_t s);
/* pt_swap_threshold for either swap rule (PT_SWAP_BARKER, PT_SWAP_METROPOLIS); all ones for
 * an unknown rule. */
uint64_t pt_swap_threshold_ex(double beta_lo, double beta_hi, int64_t n, int64_t s, int rule);

/* Library version string. */
const char* pt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PT_H_ */
