/*
 * cdl.h -- C ABI of a column-oriented Datalog engine for one GB300 GPU.
 *
 * The engine evaluates positive Horn rules H <- B1, ..., Bn (Section 2 of
 * "Column-Oriented Datalog on the GPU") to their least fixpoint.  Relations
 * are stored column-wise: one uint32 array per attribute (Section 3, the
 * decomposed storage model, with the row index as the surrogate id).  Each
 * round of the semi-naive loop (Section 3, full / delta / new versions, all
 * rules per round) runs four steps on the GPU:
 *   (a) an open-addressing hash index over the distinct values of a join
 *       column, key -> (start, count) in the relation sorted by that column
 *       (Section 3, hybrid index);
 *   (b) a join in three passes -- count each probe row's range, exclusive
 *       scan, output-partitioned write of the head columns (Algorithm 1);
 *   (c) LSD radix sort of the new tuples and removal of repeats (Section 5:
 *       per-column radix sorting);
 *   (d) set difference new - full and eager merge of the difference into the
 *       sorted full relation (Section 4, "Union and Deduplication"; Section
 *       3, "Continuous Memory Layout").
 *
 * Conventions shared by every call:
 *   - Every call returns a cdl_status; nothing aborts, asserts or traps.
 *     On error, cdl_last_error(engine) describes it (engine calls only).
 *   - Values are uint32; 0xFFFFFFFF is reserved (it marks empty hash slots)
 *     and is rejected on load with CDL_E_VALUE.
 *   - Relations are sets; loading repeats is allowed and they are dropped.
 *   - Exported tuples are unique and ordered lexicographically by unsigned
 *     column value, column 0 first.
 *   - Counts and offsets are 64-bit.  A single relation holds fewer than
 *     2^32 tuples (CDL_E_CAPACITY otherwise).
 *   - Arity is 1..CDL_MAX_ARITY.
 *   - "stream" arguments are cudaStream_t values passed as void*; NULL means
 *     the legacy default stream.  Device pointers must be 16-byte aligned.
 *   - The caller owns every buffer it passes; the library copies what it
 *     keeps.  Device memory the engine keeps comes from the caller's
 *     allocator callbacks when given, else from cudaMalloc.
 */
#ifndef CDL_H_
#define CDL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CDL_MAX_ARITY 8
#define CDL_MAX_BODY 8
#define CDL_EMPTY_KEY 0xFFFFFFFFu

typedef enum {
  CDL_OK = 0,
  CDL_E_INVALID = -1,  /* bad argument, unsupported rule shape */
  CDL_E_NOMEM = -2,    /* allocator returned NULL or the memory limit is reached */
  CDL_E_CAPACITY = -3, /* an output buffer or a 2^32 size limit is too small */
  CDL_E_VALUE = -4,    /* input holds the reserved value 0xFFFFFFFF */
  CDL_E_MAXITER = -5,  /* the fixpoint needs more rounds than max_iters */
  CDL_E_TIMEOUT = -6,  /* a bounded device-side wait ran out (no kernel of this library
                          waits on another block; the code stays reserved) */
  CDL_E_CUDA = -7,     /* a CUDA runtime call failed */
  CDL_E_STATE = -8     /* call not valid in the engine's current state */
} cdl_status;

/* ------------------------------------------------------------------------ */
/* Engine                                                                    */
/* ------------------------------------------------------------------------ */

typedef struct cdl_engine cdl_engine; /* opaque, owned by the library */
typedef uint32_t cdl_rel;

/* Device allocator supplied by the caller (e.g. backed by PyTorch).  alloc
 * returns a device pointer (>= 256-byte aligned) or NULL; free returns it. */
typedef void* (*cdl_alloc_fn)(size_t bytes, void* ctx);
typedef void (*cdl_free_fn)(void* ptr, size_t bytes, void* ctx);

typedef struct {
  cdl_alloc_fn alloc;  /* NULL: the engine uses cudaMalloc / cudaFree */
  cdl_free_fn free;
  void* alloc_ctx;
  void* stream;        /* cudaStream_t every kernel of the engine runs on */
  uint64_t mem_limit;  /* bytes of device memory the engine may hold; 0 = no limit */
  uint64_t max_iters;  /* rounds that may produce new tuples; 0 = no limit */
  uint64_t spin_limit; /* bound of any device-side wait; 0 = default (2^26).  No kernel of
                          this library spins on another block, so nothing reads it now */
  uint32_t timing;     /* CUDA-event timing of kernel launches: 0 off; 1 every kernel
                          class; any other value is a mask, bit (1 + c) timing class c
                          (the classes cdl_kernel_profile lists), so that events wrap
                          only the launches one wants timed */
  int32_t estimator;   /* join-size estimator: 0 off; 1 predict (once trained or set);
                          2 predict and log every join's features and exact size */
  double hash_load;    /* hash table load factor in (0, 0.9]; 0 = default 0.5 */
  uint32_t radix_bits; /* radix digit width 8, 9 or 10; 0 = default: 8, or 9 where 9-bit
                         digits take one pass fewer (36-bit keys: 4 passes, not 5) */
  const char* log_path; /* reserved, must be NULL */
  double est_margin;   /* predicted buffers hold 2^(prediction + est_margin) tuples;
                          0 = default 1.0 (negative values force fallbacks in tests); every
                          fallback of a run adds 0.5 for the rest of the run, up to 4 */
  uint32_t n_instances; /* > 0: batched independent fixpoints.  Column 0 of every
                           relation holds an instance id < n_instances (CDL_E_VALUE at
                           cdl_run otherwise) and every rule has one variable in column 0
                           of its head and of each body atom (CDL_E_INVALID otherwise);
                           per-instance iteration counts in cdl_stats */
  int32_t retire;       /* batched runs: 0 = default, the rows of an instance that reached
                           its fixpoint leave the merged relation until the end of the
                           run; -1 = every instance stays in it every round */
  int32_t autotune;     /* launch-parameter tuner (radix digit width and block size, hash
                           load factor): 0 off (the values above); 1 use what tune_cache
                           holds; 2 also time untried candidates (CUDA events) and write
                           the results back to tune_cache at the end of cdl_run.  Results
                           never depend on it */
  const char* tune_cache; /* tuner file path (copied at cdl_create), or NULL: in memory */
  uint64_t est_min_rows; /* joins with fewer probe rows keep the count pass (the estimator
                           skips them: there the pass is cheap); 0 = default 32768 */
  int32_t graph;        /* 1: after the first semi-naive round, run the rounds of a program
                           whose rules each join one derived atom with input relations as
                           one CUDA graph: the round captured once, repeated by a device-side
                           loop until the fixpoint (a round that outgrows the graph's buffers
                           runs on the host, then the graph is rebuilt larger); other
                           programs run as with 0.  Values >= 2: the same, with buffers
                           starting at that many rows instead of 65,536 */
  int32_t dense_bits;   /* a derived relation (not batched) whose columns need T <= dense_bits
                           bits in all keeps its new tuples of a round as a bitmap of 2^T
                           bits: join outputs set bits instead of being written, and the
                           bits read back in order are the sorted unique tuples (no radix
                           sort).  0 = default 28; -1 = never; values above 34 act as 34
                           (a 2 GB bitmap).  Results never depend on it */
  int32_t dedup;        /* step (d) of derived relations whose Full no rule variant reads
                           after round 1 (every rule naming them has no other derived body
                           atom; batched runs excluded): 0 = default, the difference and
                           merge of sorted rows; 1 = Algorithm 2 (Section 4, "Union and
                           Deduplication"): Full kept in the decomposed storage model of
                           Section 3 (rows in insertion order, per column a sorted index of
                           surrogate ids and the unique hashmap over it), a new tuple is in
                           Full when the id ranges of its values overlap, delta is appended
                           and merged into each column's sorted index; 2 = the same with a
                           hash-only index (one multimap of column 0's (value, id) entries),
                           the alternative Section 3 argues against.  Full is sorted back
                           into rows when the run ends.  No graph rounds with 1 or 2.
                           Results never depend on it */
  double plan_launch_bytes; /* with the estimator on, the first join of a rule variant builds
                           on the side that moves fewer bytes: the build side's index (none
                           when cached; a derived relation's Full on non-leading columns
                           priced at the incremental merge it reaches from its second round)
                           plus 60 bytes per probe row, each launch or host wait of an index
                           build priced as this many bytes; 0 = default 2e7 (~3 us of HBM
                           traffic).  Results never depend on it */
  uint64_t est_max_rows; /* predictions above this many output rows keep the exact count
                           pass (a redo of a large join after an overflow costs more than
                           the pass); 0 = default 2^24 */
  int32_t host_full;    /* out-of-core relations: 1 = the Full version of derived
                           relations whose Full no rule variant reads after round 1 (as for
                           dedup) lives in pinned host memory; the merge of step (d) reads
                           and writes it in place over the CPU-GPU link, so its size is
                           bounded by host memory instead of the device's (and by
                           mem_limit, which counts device memory only).  Exports and
                           checkpoints read it where it is.  Not with dedup or batched
                           runs; no graph rounds.  0 = default, Full in device memory.
                           Results never depend on it */
  int32_t star;         /* a rule whose join chain ends with two atoms that both key only on
                           variables of the probe side before them (same generation's
                           edge(a, x), sg(a, b), edge(b, y)): 0 = default, one join probes
                           both atoms' hash indexes from each probe row and writes the head
                           tuples for every pair of matched rows (count pass: the product
                           of the two range lengths), so the table of the first join's
                           results is never written (positive values act as 0); a
                           negative value = a chain of binary joins (Algorithm 1)
                           throughout.  A probe row with 2^32 or more outputs raises
                           CDL_E_CAPACITY.  Results never depend on it */
} cdl_options;

/* Fills *opts with the defaults (everything zero / NULL except the
 * defaults stated above). */
void cdl_options_default(cdl_options* opts);

/* Creates an engine on the current CUDA device.  Section 2: a program is a
 * set of rules over input (EDB) and derived (IDB) relations. */
cdl_status cdl_create(const cdl_options* opts, cdl_engine** out);

/* Frees everything the engine holds.  NULL is accepted. */
cdl_status cdl_destroy(cdl_engine* e);

/* Declares a relation of the given arity (Section 3: n-ary relations stored
 * as one column per attribute).  Names are unique. */
cdl_status cdl_relation_create(cdl_engine* e, const char* name, uint32_t arity, cdl_rel* out);

/* Adds n tuples to relation rel: cols[k] points to n uint32 values of column
 * k (host memory if on_device == 0, device memory otherwise).  The library
 * copies and checks the values; repeats are dropped.  Must precede cdl_run.
 * Returns CDL_E_VALUE if a value is 0xFFFFFFFF (nothing is added then).
 * The sort and merge into the relation happen, for every relation loaded
 * since, at the next call that reads relations (cdl_run, size, export). */
cdl_status cdl_relation_load(cdl_engine* e, cdl_rel rel, const uint32_t* const* cols,
                             uint64_t n, int on_device);

/* Loads several relations at once: the same as count calls
 * cdl_relation_load(e, rels[i], cols[i], n[i], on_device), except that the
 * values of all of them are checked together with one wait for the device.
 * Returns CDL_E_VALUE if any of them holds 0xFFFFFFFF, and then none of them
 * is added.  CDL_E_INVALID (nothing added) for a null array, an unknown
 * relation or a null column pointer. */
cdl_status cdl_relations_load(cdl_engine* e, uint32_t count, const cdl_rel* rels,
                              const uint32_t* const* const* cols, const uint64_t* n,
                              int on_device);

typedef struct {
  uint32_t is_const; /* 0: variable, 1: constant */
  uint32_t v;        /* variable id (any small integer) or constant value */
} cdl_term;

typedef struct {
  cdl_rel rel;
  uint32_t arity;
  const cdl_term* terms; /* arity terms */
} cdl_atom;

/* A Horn rule head <- body[0], ..., body[nbody-1], with nneq inequalities
 * neq[2i] != neq[2i+1] between variable ids (the x != y of Section 5.2).
 * Every head variable must occur in the body, bodies have 1..CDL_MAX_BODY
 * atoms, and consecutive atoms of the join order must share a variable.
 * The rule is lowered to copy / join / project plans (Section 4). */
typedef struct {
  cdl_atom head;
  uint32_t nbody;
  const cdl_atom* body;
  uint32_t nneq;
  const uint32_t* neq;
} cdl_rule;

cdl_status cdl_rule_add(cdl_engine* e, const cdl_rule* rule);

typedef struct {
  uint64_t iterations;     /* rounds that produced a new tuple */
  uint64_t rounds;         /* rounds executed (the last found nothing new) */
  uint64_t derived_tuples; /* sum over derived relations of their size */
  double seconds;          /* device time of the run (CUDA events) */
  double algo_bytes;       /* bytes the steps must move (see the design notes) */
  uint64_t joins;          /* join operations executed */
  uint64_t kernel_launches;
  uint64_t est_predictions; /* joins sized by the estimator */
  uint64_t est_overflows;   /* of those, joins that fell back to the exact count */
  uint64_t* delta_per_round; /* caller array or NULL: new tuples per round */
  uint64_t delta_cap;        /* its length */
  uint64_t* iters_per_instance; /* caller array of n_instances or NULL: for a batched run,
                                   the last round in which each instance derived a tuple */
  uint64_t graph_rounds;  /* options.graph: rounds run by the captured graph's device loop */
  uint64_t graph_builds;  /* options.graph: graphs captured (one more after each round that
                             outgrew the graph's buffers) */
  uint64_t index_merges;  /* indexes of a derived relation's Full sorted by non-leading key
                             columns that were updated by merging the round's delta into the
                             previous version's index (Section 3's sorted indices kept
                             incrementally) instead of sorting Full again */
  uint64_t graph_retirements; /* batched runs with options.graph: rounds of the captured
                             graph in which converged instances' rows left Full (decided and
                             moved on the device) */
  uint64_t star_joins;    /* joins that probed two atoms from each probe row (options.star) */
} cdl_stats;

/* Runs the semi-naive loop to the fixpoint on the engine's stream and waits
 * for it.  CDL_E_MAXITER if more than max_iters rounds produce tuples.
 * Rules may not be added afterwards (CDL_E_STATE). */
cdl_status cdl_run(cdl_engine* e, cdl_stats* stats);

/* Number of tuples of rel (after loads or a run). */
cdl_status cdl_relation_size(cdl_engine* e, cdl_rel rel, uint64_t* n);

/* Copies rel's tuples, sorted and unique, into cols[k] (cap tuples each;
 * host memory if on_device == 0).  *n_written receives the size; a cap
 * below the size gives CDL_E_CAPACITY and writes nothing. */
cdl_status cdl_relation_export(cdl_engine* e, cdl_rel rel, uint32_t* const* cols, uint64_t cap,
                               uint64_t* n_written, int on_device);

/* Checkpoints (not in the paper).  cdl_checkpoint_save, after cdl_run
 * returned CDL_OK or CDL_E_MAXITER, writes every relation's full and delta
 * versions and the rounds completed (with their delta sizes) to a file.
 * cdl_checkpoint_load, on a fresh engine whose relations and rules are
 * declared as before and before cdl_run, restores them: cdl_run then
 * continues the semi-naive loop from the saved round with the saved deltas
 * (iterations, rounds and per-round sizes continue the saved ones).
 * CDL_E_STATE out of order, CDL_E_INVALID for an unreadable, foreign or
 * mismatching file and for batched engines. */
cdl_status cdl_checkpoint_save(cdl_engine* e, const char* path);
cdl_status cdl_checkpoint_load(cdl_engine* e, const char* path);

/* Copies rows [first, first + count) of rel (sorted and unique, as
 * cdl_relation_export orders them) into cols[k] (count tuples each; host
 * memory if on_device == 0).  A range past the size gives CDL_E_CAPACITY
 * and writes nothing. */
cdl_status cdl_relation_export_rows(cdl_engine* e, cdl_rel rel, uint64_t first, uint64_t count,
                                    uint32_t* const* cols, int on_device);

/* Batched runs (options.n_instances > 0): the tuples of instance `instance`
 * are rows [*first, *first + *count) of rel, column 0 holding the instance
 * id.  CDL_E_INVALID for an unbatched engine or an instance id >=
 * n_instances. */
cdl_status cdl_instance_rows(cdl_engine* e, cdl_rel rel, uint32_t instance, uint64_t* first,
                             uint64_t* count);

/* Per-kernel timing gathered while options.timing != 0: for kernel class
 * idx (0..), its name, launches, summed device milliseconds and summed
 * algorithmic bytes.  CDL_E_INVALID when idx is past the last class. */
cdl_status cdl_kernel_profile(cdl_engine* e, uint32_t idx, char* name, size_t name_cap,
                              uint64_t* launches, double* ms, double* bytes);

/* Engine-owned description of the last error; valid until the next call. */
const char* cdl_last_error(const cdl_engine* e);

/* ------------------------------------------------------------------------ */
/* Learned join-size estimator (not in the paper; see the design notes)      */
/* ------------------------------------------------------------------------ */
/* A 16 -> 64 -> 64 -> 1 ReLU network predicts log2(1 + join size) from 16
 * features of each join (sizes, sampled distinct keys, 32-bucket key-hash
 * histograms of both sides, round, previous sizes, filter flag).  With a
 * trained network and options.estimator >= 1 the engine sizes each join's
 * output buffer at 2^(prediction + est_margin) tuples, writes the join in
 * one pass without Algorithm 1's count and scan, and falls back to the exact
 * three-pass join when the buffer overflows.  Results never depend on it.
 * Parameters: CDL_MLP_PARAMS floats, W1 (64x16 row-major), b1 (64), W2
 * (64x64 row-major), b2 (64), w3 (64), b3 (1). */
#define CDL_MLP_IN 16
#define CDL_MLP_PARAMS 5313

/* Copies the logged samples (options.estimator == 2: one per join the
 * engine ran) into X (n x 16, row-major) and y (log2(1 + exact size)), at
 * most cap; *n receives the number logged.  X / y may be NULL to query. */
cdl_status cdl_estimator_log(cdl_engine* e, float* X, float* y, uint64_t cap, uint64_t* n);

/* Trains the network on the GPU from He-uniform weights drawn with seed:
 * `epochs` full-batch Adam steps (learning rate lr) on the pinball loss at
 * level tau (e.g. 0.9, so that predictions err on the large side), over the
 * n host samples X / y, or over the engine's own log when X is NULL.
 * *loss (may be NULL) receives the final training loss.  The engine then
 * predicts with the trained network (BF16 copy). */
cdl_status cdl_estimator_train(cdl_engine* e, const float* X, const float* y, uint64_t n,
                               uint32_t epochs, float lr, float tau, uint64_t seed, float* loss);

/* Reads (set == 0) or installs (set == 1) the network's FP32 parameters
 * (host array of CDL_MLP_PARAMS floats). */
cdl_status cdl_estimator_params(cdl_engine* e, float* params, int set);

/* Network steps on caller-owned device buffers (FP32 parameters, inputs
 * X n x 16 row-major), for tests and tools; workspace protocol as below. */
cdl_status cdl_mlp_forward(const float* params, const float* X, uint64_t n, float* out,
                           void* workspace, size_t* ws_bytes, void* stream);
/* FP32 forward + backward: out = predictions, grad = d(mean pinball loss at
 * level tau)/d(params) over the n samples. */
cdl_status cdl_mlp_gradient(const float* params, const float* X, const float* y, uint64_t n,
                            float tau, float* out, float* grad, void* workspace, size_t* ws_bytes,
                            void* stream);
/* Inference with the parameters rounded to BF16, BF16 activations, FP32
 * accumulation (the engine's prediction path). */
cdl_status cdl_mlp_infer_bf16(const float* params, const float* X, uint64_t n, float* out,
                              void* workspace, size_t* ws_bytes, void* stream);
/* One Adam step (Kingma & Ba, 2015: b1 = 0.9, b2 = 0.999, eps = 1e-8, bias
 * correction with step counted from 1) of the network's training, on
 * caller-owned device arrays of CDL_MLP_PARAMS floats: params is updated in
 * place from grad; m and v are the first and second moment estimates (zero
 * before step 1), updated in place.  CDL_E_INVALID on a NULL array or
 * step 0.  Asynchronous on stream. */
cdl_status cdl_mlp_adam(float* params, const float* grad, float* m, float* v, uint64_t step,
                        float lr, void* stream);

/* The 16 input features of one join, written as floats to the device array
 * features (the learned estimator is not in the paper; the features read
 * "delta/full sizes, sampled distinct counts and 32-bucket key histograms"):
 * a deterministic stride sample of at most 2048 join keys per side (sample
 * s of n keys is key s * n / min(n, 2048)); each key hashed with the
 * MurmurHash3 finaliser, h = fmix32(k0 ^ fmix32(k1 + 0x9e3779b9)), k1 = 0
 * for one-column keys, bucketed by the hash's top 5 bits; distinct counts
 * of sampled hashes.  probe_k0 / build_k0: device key columns of n_probe /
 * n_build rows; probe_k1 / build_k1: second key columns or NULL.  host: 6
 * host floats {|full| of the probe relation, distinct build keys, round,
 * previous exact output of the step, previous delta of the head relation,
 * 1 if the step filters else 0}.  Features, in order: log2(1 + x) of probe
 * rows, build rows, host[0], distinct sampled probe / build hashes, build
 * rows / max(1, host[1]); log2(1 + histogram join estimate); largest
 * bucket share (probe, build); bucket entropy in bits (probe, build);
 * cosine of the two histograms; host[2]; log2(1 + host[3]);
 * log2(1 + host[4]); host[5].  Asynchronous on stream. */
cdl_status cdl_join_features(const uint32_t* probe_k0, const uint32_t* probe_k1, uint64_t n_probe,
                             const uint32_t* build_k0, const uint32_t* build_k1, uint64_t n_build,
                             const float* host, float* features, void* stream);

/* ------------------------------------------------------------------------ */
/* Steps of one round on caller-owned device buffers                          */
/* ------------------------------------------------------------------------ */
/* These run exactly the kernels the engine uses, on plain device pointers.
 * Scratch memory comes from the caller: each call with workspace == NULL
 * only reports the bytes it needs in *ws_bytes and returns CDL_OK. */

/* Bytes of a hash table for n_keys distinct keys at load factor load
 * (slots are 16 bytes, the slot count a power of two). */
uint64_t cdl_hash_table_bytes(uint64_t n_keys, double load);

/* Step (a), Section 3 hybrid index.  keys: n values sorted ascending.  For
 * every distinct value v the table receives (v, start, count): the first
 * position of v in keys and its run length.  table_bytes must be at least
 * cdl_hash_table_bytes(n, load) for some load <= 0.9 (so that every key
 * finds a slot); CDL_E_INVALID otherwise. */
cdl_status cdl_hash_build(const uint32_t* keys, uint64_t n, void* table, uint64_t table_bytes,
                          void* stream);

/* Step (b) first pass, Algorithm 1 probe loop: counts[i] = number of
 * occurrences of probe[i] in the table's column (0 if absent). */
cdl_status cdl_join_count(const uint32_t* probe, uint64_t n, const void* table,
                          uint64_t table_bytes, uint32_t* counts, void* stream);

/* Step (b) second pass: out[i] = sum of in[0..i) in 64 bits; *total_host
 * (host pointer, may be NULL) receives the sum of all n (the call then waits
 * for the stream). */
cdl_status cdl_exclusive_scan(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* total_host,
                              void* workspace, size_t* ws_bytes, void* stream);

/* The same scan as cdl_exclusive_scan for callers that cannot allocate
 * device memory (no cudaMalloc, no workspace to hand over): it allocates
 * nothing.  The paper has no counterpart; this is a convenience of this
 * library.  Its scratch is a fixed array inside the library, 512 KiB + 8
 * bytes on every GPU where the library is loaded, held until the process
 * exits; so n may not exceed 134,217,728 (65,536 tiles of 2048), and larger
 * n gives CDL_E_CAPACITY with nothing launched.  The first call on each GPU
 * looks up the array's device address (with that GPU current); make that
 * first call before any stream capture.  All calls share the one array:
 * calls whose kernels overlap on the GPU (other streams, other threads)
 * race on it and must be serialised by the caller.  Every value the scan
 * reads from the array is written by the same call first.  Arguments and
 * results as for cdl_exclusive_scan. */
cdl_status cdl_exclusive_scan_noalloc(const uint32_t* in, uint64_t n, uint64_t* out,
                                      uint64_t* total_host, void* stream);

/* Where a head column of a join takes its value from. */
typedef struct {
  uint32_t side; /* 0: probe row column, 1: build row column, 2: constant */
  uint32_t v;    /* column index, or the constant */
} cdl_colref;

/* Step (b) complete (hash build on the build side + count + scan + write,
 * Algorithm 1 with output partitioning, projection fused).  The build side
 * must be sorted by build_cols[build_key].  For every probe row p and build
 * row b with probe_cols[probe_key][p] == build_cols[build_key][b] and
 * column(neq[2i]) != column(neq[2i+1]) for every inequality, one output
 * tuple out[k] = value of spec[k] is written.  Without inequalities the
 * output is in Algorithm 1's order (probe row, then build position); with
 * them, surviving tuples are packed in an unspecified order.  *n_out
 * receives the tuple count; out_cap below the unfiltered join size gives
 * CDL_E_CAPACITY with *n_out = that size and nothing written. */
cdl_status cdl_join(const uint32_t* const* probe_cols, uint32_t probe_arity, uint64_t n_probe,
                    uint32_t probe_key, const uint32_t* const* build_cols, uint32_t build_arity,
                    uint64_t n_build, uint32_t build_key, const cdl_colref* spec, uint32_t out_arity,
                    const cdl_colref* neq, uint32_t nneq, uint32_t* const* out_cols,
                    uint64_t out_cap, uint64_t* n_out, void* workspace, size_t* ws_bytes,
                    void* stream);

/* Step (c): sorts n tuples of arity columns lexicographically (LSD radix
 * sort, stable), drops repeats, writes the unique tuples to out_cols and
 * their number to *n_out.  cols are left unchanged. */
cdl_status cdl_sort_unique(const uint32_t* const* cols, uint32_t arity, uint64_t n,
                           uint32_t* const* out_cols, uint64_t* n_out, void* workspace,
                           size_t* ws_bytes, void* stream);

/* Step (d): full (n_full tuples) is sorted and unique; fresh (n_fresh tuples)
 * is sorted, repeats allowed.  Writes delta = fresh - full (sorted, unique,
 * *n_delta tuples) and merged = full U delta (sorted, n_full + *n_delta
 * tuples).  merged must hold n_full + n_fresh tuples, delta n_fresh. */
cdl_status cdl_diff_merge(const uint32_t* const* full, uint64_t n_full,
                          const uint32_t* const* fresh, uint64_t n_fresh, uint32_t arity,
                          uint32_t* const* delta, uint64_t* n_delta, uint32_t* const* merged,
                          void* workspace, size_t* ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CDL_H_ */
