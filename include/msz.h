/*
 * msz.h: C ABI of the GB300 MSz correction library (libmsz.so).
 *
 * MSz (Li et al., "MSz: An Efficient Parallel Algorithm for Correcting
 * Morse-Smale Segmentations in Error-Bounded Lossy Compressors") edits a
 * decompressed scalar field fhat until the piecewise-linear Morse-Smale
 * segmentation of the edited field g equals that of the original f, while
 * every value stays within the absolute error bound xi (Sec. 3, "Problem
 * Statement": |f_i - g_i| <= xi, M = Mhat, m = mhat). The edits are
 * returned as a list of (vertex index, new value) pairs (Sec. 5.3) that
 * msz_apply() writes into fhat on the decompression side (Fig. 3).
 *
 * Conventions shared by every entry point:
 *   - Fields are dense 2D or 3D grids, x fastest: vertex (x, y, z) has the
 *     linear index x + nx*(y + ny*z). dims[] = {nx, ny, nz}; for ndim == 2
 *     dims[2] is ignored. Every extent is >= 1 and nx*ny*nz < 2^31.
 *   - The mesh is the Freudenthal triangulation of the grid: the neighbours
 *     of v are v + e and v - e for every nonzero e in {0,1}^ndim that stays
 *     inside the grid (6 in 2D, 14 in 3D).
 *   - Ties between equal values are broken by the linear index (the
 *     simulation of simplicity of Sec. 3); IEEE comparison, so -0 == +0.
 *   - xi is rounded once to the field's type; the lower bound of vertex i is
 *     the smallest representable value >= f_i - xi.
 *   - Pointers named *_dev are device pointers on the current CUDA device;
 *     *_host are host pointers (pageable or pinned). Input buffers are
 *     borrowed: they must stay valid and unmodified until the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Every call returns when its results are ready.
 *   - Errors are negative msz_status codes; no C++ exception crosses the ABI.
 *     msz_strerror() names them.
 */
#ifndef MSZ_H_
#define MSZ_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { MSZ_F32 = 0, MSZ_F64 = 1 } msz_dtype;

typedef enum {
  MSZ_OK = 0,
  MSZ_ERR_ARG = -1,        /* bad argument: ndim, dims, NULL pointer, xi < 0 or not finite,
                              or a lower bound f - xi that overflows */
  MSZ_ERR_DTYPE = -2,      /* dtype is neither MSZ_F32 nor MSZ_F64 */
  MSZ_ERR_NONFINITE = -3,  /* f or fhat holds a NaN or an infinity */
  MSZ_ERR_BOUND = -4,      /* fhat violates |fhat - f| <= xi at some vertex */
  MSZ_ERR_OOM = -5,        /* device or host allocation failed */
  MSZ_ERR_NOCONVERGE = -6, /* round cap reached (msz_options.max_rounds); the result still
                              holds the edit list of the field after its last round; its label
                              arrays hold f's labels, which g's do not match yet */
  MSZ_ERR_TIMEOUT = -7,    /* a bounded device-side wait gave up */
  MSZ_ERR_CUDA = -8,       /* a CUDA runtime call failed */
  MSZ_ERR_BUSY = -9,       /* server: no free slot / request id unknown or not finished */
  MSZ_ERR_TOO_LARGE = -10, /* msz_fix_noalloc: the field does not fit its static scratch */
  MSZ_ERR_CANCELLED = -11, /* server: the request was cancelled (msz_server_cancel) */
  MSZ_ERR_CHECK = -12      /* checked build only (libmsz_checked.so, compiled with MSZ_CHECKED):
                              an index read from device data was out of range; the access was
                              skipped and the fix stopped being meaningful */
} msz_status;

/* Counters of one fix. The same quantities are computed by the reference
 * restatement of the method, so they are compared exactly in the tests. */
typedef struct {
  uint64_t sweeps;       /* evaluations of directions of a changed field */
  uint64_t c_rounds[4];  /* C-loop edit rounds: FPmax, FPmin, FNmax, FNmin (Sec. 4.1) */
  uint64_t c_cases[4];   /* false critical points edited, summed over those rounds */
  uint64_t c_passes;     /* completed passes over the four C sub-loops */
  uint64_t r_rounds;     /* R-loop edit rounds (Sec. 4.2) */
  uint64_t r_cases[2];   /* troublemakers edited: wrong max label, wrong min label */
  uint64_t label_evals;  /* max/min label computations of g */
  uint64_t mismatch[2];  /* wrong max / min labels, summed over label computations */
  uint64_t dec_edits;    /* decreasing edits applied (Eqs. 2-6) */
  uint64_t freezes;      /* vertices reset to f by the termination guard */
  uint64_t edits;        /* length of the final edit list */
  /* Requests that froze their anchor's closed ring instead of decreasing
   * their target (the termination guard), by the case that made them:
   * C-loop FPmax, FPmin, FNmax, FNmin, R-loop wrong max label, wrong min
   * label. freeze_req counts them all, freeze_req_frozen those whose target
   * was already frozen; the others found the target at its lower bound. */
  uint64_t freeze_req[6];
  uint64_t freeze_req_frozen[6];
} msz_counts;

/* msz_options.flags */
#define MSZ_OPT_NO_TMA 1u        /* stage sweep planes with plain loads instead of TMA */
#define MSZ_OPT_TIME_KERNELS 2u  /* fill msz_result.kernel_ms (CUDA events around each kernel kind) */
#define MSZ_OPT_TEST_STALL 4u    /* test hook: fields start in a stage that no kernel serves, so no
                                    state machine moves and the host's stall detection ends the
                                    fix with MSZ_ERR_TIMEOUT (nothing waits or spins on the device) */

typedef struct {
  uint64_t max_rounds;   /* cap on C + R edit rounds; 0 = default (10^7). A fix that applies
                            round max_rounds + 1 stops there with MSZ_ERR_NOCONVERGE */
  int32_t  autotune;     /* batches: nonzero = the first msz_batch_fix first runs
                            msz_batch_autotune on its inputs (plans: ignored) */
  uint32_t flags;        /* MSZ_OPT_* bits */
  int32_t  reserved[6];
} msz_options;

/* Launch parameters of the correction loop (no counterpart in the paper:
 * they decide how the work is scheduled on the GPU, never what is computed;
 * every valid setting gives bit-identical results). */
typedef struct {
  int32_t jumps_per_step;  /* label propagation launches per loop step, 1-4 (default 2) */
  int32_t chase_steps;     /* exit-table steps an entry follows per propagation launch, 4-256 (32) */
  int32_t small_rounds;    /* C-loop rounds one thread-block cluster launch may run, 0-1024; 0 = every
                              round on the grid kernels (64) */
  int32_t small_cases;     /* largest round (cases) the cluster takes, 1-65536 (65536) */
  int32_t graph_steps;     /* loop steps per captured CUDA graph, 1-8 (4) */
  int32_t sweep_chunk;     /* planes per tile of the full classification sweep, 4-64 (64) */
  int32_t blocks_per_sm;   /* blocks per SM of the grid-wide kernels, at most their occupancy;
                              0 = their occupancy (0) */
  int32_t reserved[5];     /* zero */
} msz_tuning;

/* Fills *t with the defaults above. */
void msz_tuning_default(msz_tuning* t);
/* MSZ_OK if every field of *t is in range, else MSZ_ERR_ARG (host only). */
int msz_tuning_valid(const msz_tuning* t);

/* Results of msz_fix / msz_fix_host. For msz_fix the arrays are DEVICE
 * memory owned by the plan: valid until the next msz_fix on that plan or
 * msz_plan_destroy. For msz_fix_host they are the caller's host buffers. */
typedef struct {
  uint32_t* edit_idx;    /* n_edits vertex indices, strictly ascending */
  void*     edit_val;    /* n_edits new values, the field's type */
  uint64_t  n_edits;
  int32_t*  label_max;   /* N labels: index of the maximum each vertex ascends to */
  int32_t*  label_min;   /* N labels: index of the minimum each vertex descends to */
  msz_counts counts;
  int32_t   status;      /* msz_status of the fix */
  float     device_ms;   /* device time of the fix (CUDA events), 0 if not timed */
  uint64_t  launches;    /* kernels this library launched for the fix */
  float     kernel_ms[4];/* with MSZ_OPT_TIME_KERNELS: summed device time of the C-loop sweep,
                            label pointer jumping, R-loop check, and mark + apply kernels */
} msz_result;

typedef struct msz_plan_s* msz_plan;

/* Allocates the device state for fields of one shape and type (Sec. 4 state:
 * g, directions, labels of f and g, per-vertex flags, case and edit lists).
 * opt may be NULL. Returns MSZ_ERR_OOM if device memory is insufficient and
 * MSZ_ERR_CUDA if no CUDA device can be used. */
int msz_plan_create(msz_plan* out, int ndim, const int64_t dims[3], int dtype,
                    const msz_options* opt);

/* Device bytes a plan of this shape and type allocates (for admission). */
int64_t msz_plan_bytes(int ndim, const int64_t dims[3], int dtype);

int msz_plan_destroy(msz_plan p);

/* Per-kernel statistics of the last msz_fix on a plan created with
 * MSZ_OPT_TIME_KERNELS (no counterpart in the paper: instrumentation). Every
 * launch of a loop step is bracketed by CUDA events; a launch "works" when it
 * completes a stage of the field's state machine (the others find the field
 * in another stage and return at once). units counts the work of the working
 * launches: vertices (k_csweep), algorithmic bytes (k_label_tile: per
 * vertex of a recomputed tile 5 in g's passes, 14 in f's, and 16 per face
 * cell of every tile for the exit tables' entries; k_rcheck: 8 per exit
 * label looked up, 12 per vertex of the tiles examined), exit-table
 * accesses (k_jump), cases (k_gather, k_mark),
 * touched vertices (k_apply), ring items (k_reclass), C-loop rounds run
 * whole in one thread-block cluster per field (k_csmall: requests, apply and
 * reclassification of rounds with few cases). */
#define MSZ_NUM_KERNELS 9
typedef struct {
  const char* name;        /* kernel name, static string */
  uint64_t launches;       /* launches inside the loop's steps */
  uint64_t work_launches;  /* of which did work for the field */
  double ms;               /* device time of all launches */
  double work_ms;          /* device time of the working launches */
  uint64_t units;          /* work units of the working launches (see above) */
} msz_kernel_stat;

/* Fills out[0 .. min(n, MSZ_NUM_KERNELS) - 1] in the order k_csweep,
 * k_gather, k_mark, k_label_tile, k_jump, k_rcheck, k_apply, k_reclass,
 * k_csmall;
 * returns the number filled, or MSZ_ERR_ARG (no plan / out, or a plan made
 * without MSZ_OPT_TIME_KERNELS). Host memory only. */
int msz_plan_kernel_stats(msz_plan p, msz_kernel_stat* out, int n);

/* The correction loop (Sec. 4, Fig. 3 top): given the original field f and
 * the decompressed field fhat (device, N values of the plan's type) and the
 * bound xi, runs C-loops and R-loops until no false critical point and no
 * wrong label is left, entirely on the device. Fills *out (device arrays
 * owned by the plan). Returns out->status. */
int msz_fix(msz_plan p, const void* orig_dev, const void* decomp_dev, double xi,
            void* stream, msz_result* out);

/* Same loop from host buffers: copies f and fhat to the plan's device
 * buffers, runs msz_fix, and copies the edit list (and, if label_max_host /
 * label_min_host are non-NULL, the labels) back. edit_idx_host / edit_val_host
 * must hold N entries (the worst case). out->edit_idx / edit_val / label_*
 * are set to the host buffers. */
int msz_fix_host(msz_plan p, const void* orig_host, const void* decomp_host, double xi,
                 uint32_t* edit_idx_host, void* edit_val_host, int32_t* label_max_host,
                 int32_t* label_min_host, void* stream, msz_result* out);

/* Batched form: many independent fields of uneven shapes and mixed
 * float32 / float64 corrected together (Sec. 5's per-vertex parallelism
 * applied across fields). The fields of each (dtype, dimension) class are
 * dealt in turn to two groups; every kernel of a step works on all fields of
 * a group at once, and the groups run their steps concurrently on streams of
 * their own, forked from and joined back into `stream`. Each field keeps its
 * own state machine and drops out when it converges, so the results are
 * bit-identical to msz_fix on each field alone. The step sequence is
 * captured once in a CUDA graph and replayed.
 *   n fields; ndim[i], dims[3*i .. 3*i+2], dtype[i] as for msz_plan_create.
 *   msz_batch_fix: orig_dev[i], decomp_dev[i], xi[i] per field; results[i]
 *   receives field i's result (device arrays owned by the batch, valid until
 *   the next msz_batch_fix or msz_batch_destroy). Returns MSZ_OK when every
 *   field succeeded, else the first failing field's status. */
typedef struct msz_batch_s* msz_batch;
int64_t msz_batch_bytes(int n, const int* ndim, const int64_t* dims, const int* dtype);
int msz_batch_create(msz_batch* out, int n, const int* ndim, const int64_t* dims, const int* dtype,
                     const msz_options* opt);
int msz_batch_fix(msz_batch b, const void* const* orig_dev, const void* const* decomp_dev, const double* xi,
                  void* stream, msz_result* results);
int msz_batch_destroy(msz_batch b);

/* Launch parameters of a batch (or plan): set (validated; takes effect at
 * the next fix) and read. */
int msz_batch_set_tuning(msz_batch b, const msz_tuning* t);
int msz_batch_get_tuning(msz_batch b, msz_tuning* t);
int msz_plan_set_tuning(msz_plan p, const msz_tuning* t);
int msz_plan_get_tuning(msz_plan p, msz_tuning* t);

/* Autotuner of the batched form: times the batch on these inputs under the
 * current launch parameters and under candidates for one parameter at a time
 * (coordinate descent over jumps_per_step, chase_steps, small_rounds,
 * small_cases, graph_steps, sweep_chunk, blocks_per_sm; two timed fixes per
 * candidate, the faster counts), keeps a candidate only when it is faster by
 * more than 2%, and applies the best setting to the batch. The result is
 * cached for the process under a signature of the batch (per field: dtype,
 * dimension and log2 of the vertex count); a batch with a cached signature
 * takes the cached setting without timing unless force is nonzero. *out
 * receives the applied setting, *tried (nullable) the number of settings
 * timed. Results of later fixes are identical to untuned ones. */
int msz_batch_autotune(msz_batch b, const void* const* orig_dev, const void* const* decomp_dev, const double* xi,
                       int force, void* stream, msz_tuning* out, int* tried);

/* Served form: continuous batching. A worker thread owned by the server
 * admits submitted fields while slots (max_slots) and device memory
 * (budget_bytes, counted with msz_plan_bytes) allow, and corrects all
 * resident fields together, step by step, each with its own state machine
 * kept on the device until it converges; fields that arrive while others are
 * running join at the next chunk of steps. Results equal msz_fix on each
 * field alone.
 *   msz_server_submit: inputs must be ready on the device and stay valid and
 *     unmodified until the request finishes; returns a request id at once.
 *   msz_server_poll: waits up to wait_ms; MSZ_OK when finished (out filled:
 *     out->status is the field's status, out->device_ms the submit-to-result
 *     latency, arrays are device memory held until msz_server_release),
 *     MSZ_ERR_BUSY while queued or running, MSZ_ERR_ARG for an unknown id.
 *     A field larger than the whole budget finishes with MSZ_ERR_OOM.
 *   msz_server_release: frees a finished request's memory.
 *   msz_server_destroy: stops the worker; running requests are abandoned. */
typedef struct msz_server_s* msz_server;
int msz_server_create(msz_server* out, int64_t budget_bytes, int max_slots, const msz_options* opt);
int msz_server_submit(msz_server s, int ndim, const int64_t dims[3], int dtype, const void* orig_dev,
                      const void* decomp_dev, double xi, uint64_t* request_id);
int msz_server_poll(msz_server s, uint64_t request_id, int wait_ms, msz_result* out);
int msz_server_release(msz_server s, uint64_t request_id);
/* Cancels a request (host side; no device wait is involved). A queued
 * request is dropped at once; a running one leaves the running set at the
 * next chunk boundary, when none of the server's kernels is in flight, and
 * the other resident fields go on unchanged. Either way the request then
 * finishes with status MSZ_ERR_CANCELLED (msz_server_poll) and is released
 * as usual. MSZ_ERR_BUSY if it already finished, MSZ_ERR_ARG for an unknown
 * id. */
int msz_server_cancel(msz_server s, uint64_t request_id);
int msz_server_destroy(msz_server s);

/* Decompression side (Fig. 3 bottom; g_i = fhat_i + delta_i, Sec. 3):
 * writes edit_val[k] into decomp_dev[edit_idx[k]] for k < n_edits. Indices
 * must be < N (checked on the device: out-of-range entries are skipped and
 * MSZ_ERR_ARG is returned). n_edits == 0 is a no-op. */
int msz_apply(void* decomp_dev, int ndim, const int64_t dims[3], int dtype,
              const uint32_t* edit_idx_dev, const void* edit_val_dev, uint64_t n_edits,
              void* stream);

/* Directions of one field (the per-vertex step of Sec. 5.1 "Updating
 * directions"): dir_dev[v] = ascending slot | descending slot << 4, where a
 * slot s < 14 is the neighbour v + e_s (e_0..e_6 = (1,0,0), (0,1,0), (0,0,1),
 * (1,1,0), (1,0,1), (0,1,1), (1,1,1); e_7..e_13 their negations; in 2D
 * e_0..e_2 = (1,0), (0,1), (1,1) and e_3..e_5 their negations) and 15 is v
 * itself (a maximum, resp. minimum). */
int msz_directions(const void* field_dev, int ndim, const int64_t dims[3], int dtype,
                   uint8_t* dir_dev, void* stream);

/* Evaluation metrics of a field g against the original f (the paper's
 * Appendix B: PSNR and the right labelled ratio; no counterpart in the
 * correction loop). f_dev and g_dev are device arrays of one shape and dtype,
 * x fastest. In double precision:
 *   mse            = (1/N) sum_i (f_i - g_i)^2
 *   value_range    = max_i f_i - min_i f_i          (the peak signal value)
 *   psnr           = 20 log10(value_range / sqrt(mse)), +inf when mse = 0
 *   wrong          = vertices whose maximum or minimum label (Sec. 3) under g
 *                    differs from the one under f
 *   right_labelled = 1 - wrong / N
 * The labels come from dense pointer doubling over the field, independent of
 * the correction loop's labelling. Allocates 16 bytes per vertex of stream-
 * ordered scratch for the call and returns once the results are in *out.
 * Returns MSZ_OK, MSZ_ERR_ARG (shape, NULL pointer), MSZ_ERR_DTYPE,
 * MSZ_ERR_OOM, MSZ_ERR_TIMEOUT (no fixed point within 64 rounds: cannot
 * happen for finite fields) or MSZ_ERR_CUDA. */
typedef struct {
  double mse;
  double value_range;
  double psnr;
  double right_labelled;
  uint64_t wrong;
} msz_metric_values;
int msz_field_metrics(const void* f_dev, const void* g_dev, int ndim, const int64_t dims[3], int dtype,
                      void* stream, msz_metric_values* out);

/* Lossless coding of an edit list (Sec. 5.3: the ascending indices as
 * differences with run-length and Huffman coding; the values coded
 * separately). Encoding and decoding run on the device. Format
 * (little-endian bytes):
 *   header, 14 u32 words: magic 0x45535A4D ('MSZE'), version 1, dtype,
 *     bytes per value, n_edits (u64), index tokens, index chunks, value
 *     chunks, 0, index payload bits (u64), value payload bits (u64);
 *   256 code lengths of the index symbols, 256 of the value symbols (u8,
 *     0 = unused, at most 15);
 *   per index chunk: bit offset (u64), first edit (u32), index before it
 *     (u32, 0xffffffff for none); per value chunk: bit offset (u64);
 *   the index payload, then the value payload, in u32 words, bits most
 *     significant first.
 * Index symbols, per edit k with delta d = idx[k] - idx[k-1] (idx[-1] = -1),
 * within aligned groups of 32 edits: a maximal run of L >= 2 deltas equal to
 * 1 in the group is symbol 252 followed by 5 raw bits (L - 2); otherwise
 * symbol d - 1 (d <= 252), symbol 253 + 16 raw bits (d - 253, d <= 65788) or
 * symbol 254 + 32 raw bits (d). Value symbols: the bytes of bits(value) XOR
 * bits(fhat[idx]), little-endian, per edit. Each stream has a canonical
 * code (symbols ordered by (length, symbol)) with lengths from package-merge
 * (optimal among codes of at most 15 bits; leaves sorted by (count, symbol),
 * a leaf before a package of equal weight). A chunk starts at every 4096th
 * symbol of a stream.
 *
 * msz_edits_encoded_bound: bytes that suffice for any list of n_edits.
 * msz_encode_edits: edit_idx_dev strictly ascending and below the field's N,
 *   edit_val_dev the new values, fhat_dev the field they replace (device);
 *   writes at most out_cap bytes to out_dev and their count to *out_bytes.
 *   MSZ_ERR_ARG for unsorted or out-of-field indices or too small a buffer.
 * msz_decode_edits: the inverse, given the same fhat; writes *n_edits
 *   indices and values (at most cap_edits). MSZ_ERR_ARG for a stream that is
 *   malformed, of another type or field size, or longer than cap_edits; the
 *   decoder bounds every index it writes or reads.
 * Both return when the results are in place (they allocate stream-ordered
 * scratch: about 36 bytes per edit plus 13 per value byte to encode). */
int64_t msz_edits_encoded_bound(uint64_t n_edits, int dtype);
int msz_encode_edits(const uint32_t* edit_idx_dev, const void* edit_val_dev, uint64_t n_edits, const void* fhat_dev,
                     int ndim, const int64_t dims[3], int dtype, void* out_dev, uint64_t out_cap,
                     uint64_t* out_bytes, void* stream);
int msz_decode_edits(const void* in_dev, uint64_t in_bytes, const void* fhat_dev, int ndim, const int64_t dims[3],
                     int dtype, uint32_t* edit_idx_dev, void* edit_val_dev, uint64_t cap_edits, uint64_t* n_edits,
                     void* stream);

/* msz_fix without any device allocation. The paper has no counterpart: this
 * entry point serves callers that cannot call cudaMalloc (a framework whose
 * allocator must not grow, a real-time loop where an allocation may block or
 * fail, a plugin whose host forbids allocation during a call).
 *
 * Inputs (orig_dev, decomp_dev: N values) and outputs are the caller's
 * device buffers: edit_idx_dev / edit_val_dev hold N entries (worst case),
 * label_max_dev / label_min_dev hold N labels. out->edit_idx etc. point to
 * them (the label buffers hold f's labels during the call). Every
 * other array of the loop lives in one static device array of 64 MiB that
 * each GPU loading the library holds until exit; a field needs about 33
 * bytes per vertex (float32, 3D; 26 in 2D) or 37 (float64, 3D; 30 in 2D) of
 * it, so up to about 2.0 M (float32) / 1.79 M (float64) vertices in 3D.
 * Larger fields are rejected with MSZ_ERR_TOO_LARGE before any work. The
 * first call on a device (and the first after the device's context was
 * reset) looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture. All calls share
 * the array: calls that overlap on the GPU race and must be serialised by
 * the caller. No timing (device_ms = 0). Returns out->status. */
int msz_fix_noalloc(int ndim, const int64_t dims[3], int dtype, const void* orig_dev,
                    const void* decomp_dev, double xi, uint32_t* edit_idx_dev, void* edit_val_dev,
                    int32_t* label_max_dev, int32_t* label_min_dev, void* stream, msz_result* out);

const char* msz_strerror(int status);

/* Library version string. */
const char* msz_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MSZ_H_ */
