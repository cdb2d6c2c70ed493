/*
 * tn.h -- C ABI of a single-GPU (sm_103a) sliced tensor-network contractor for
 * random-quantum-circuit amplitudes, after arXiv 2111.01066
 * ("Redefining the Quantum Supremacy Baseline With a New Generation Sunway
 * Supercomputer").
 *
 * The problem, in the paper's terms:
 *   - a circuit amplitude <x|U|0...0> is the contraction of a tensor network in
 *     which gates are rank-2 / rank-4 tensors and the initial state and the
 *     target basis are rank-1 tensors (SI, TN section, figure S2);
 *   - the network is contracted pairwise along an order (a list of two-tuples)
 *     found on the host (SI, TN section);
 *   - index slicing fixes a set of wires so that the network is a sum of 2^S
 *     smaller networks, each contracted alone (main text, section II);
 *   - leaving k qubits open yields 2^k correlated amplitudes in one run (main
 *     text, section III);
 *   - the linear XEB fidelity follows from amplitudes (main text, Eq. (1)).
 *
 * Conventions used by every call:
 *   - qubit q is bit q of a uint64_t; n_qubits <= 64;
 *   - the index of an amplitude inside a batch is sum_j b(open_j) 2^j over the
 *     open qubits in ascending order; bits of a closed bitstring at open
 *     positions are ignored;
 *   - a wire is labelled (q, t) = "qubit q after its t-th gate", t = 0 being the
 *     input wire;
 *   - slice id s fixes the j-th sliced wire of a plan to bit j of s;
 *   - amplitudes crossing the ABI are interleaved complex128 (re, im doubles).
 *
 * Every call returns a tn_status; 0 is success.  On failure
 * tn_last_error() returns a message for the calling thread's last failure.  No
 * C++ exception crosses this boundary.  Errors found by device kernels after an
 * asynchronous launch (a bounded wait that ran out, a violated bound) are
 * sticky on the plan: they are returned by the plan's next call and by
 * tn_plan_sync().  Calls without a plan (tn_contract_pair,
 * tn_contract_pair_noalloc, tn_selftest_bounded_wait) record such errors in a
 * per-device word that tn_device_sync() reads and clears.
 *
 * Streams are passed as `void*` holding a cudaStream_t (NULL = legacy default
 * stream) so that this header needs no CUDA include.
 *
 * Concurrency: a plan is used by one host thread at a time; different plans may
 * run on different streams.  tn_contract_pair, tn_xeb and tn_frugal_sample
 * share one small per-device scratch area (result word, error word, B' images
 * of tn_contract_pair, grown on demand), so calls of these that may overlap on
 * the same device -- from several host threads, or queued on streams that run
 * concurrently -- must be serialised by the caller.
 */
#ifndef TN_GB300_H
#define TN_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int tn_status;
#define TN_OK               0
#define TN_ERR_ARG         -1  /* invalid argument, size or range */
#define TN_ERR_OOM         -2  /* device or host allocation failed */
#define TN_ERR_CUDA        -3  /* a CUDA runtime call failed */
#define TN_ERR_PLAN        -4  /* no plan satisfies the options (e.g. the bound) */
#define TN_ERR_TIMEOUT     -5  /* a bounded device wait expired; the kernel returned early */
#define TN_ERR_UNSUPPORTED -6  /* valid request this build does not implement */
#define TN_ERR_DEVICE      -7  /* a device-side check failed (bounds, layout) */

/* Message for the calling thread's last failing call ("" if none).  The
 * pointer stays valid until the thread's next failing call. */
const char* tn_last_error(void);

/* ---------------------------------------------------------------- circuit */

/* A gate list in time order, initial state |0...0> (SI, "Random quantum
 * circuits").  gate_qubits[2g], gate_qubits[2g+1] are the qubits of gate g, the
 * second one -1 for a single-qubit gate.  gate_matrices holds the matrices of
 * all gates back to back as interleaved complex128, row-major, row = output:
 * 4 complex entries for a single-qubit gate, 16 for a two-qubit gate, whose
 * row/column index is 2*b(q0) + b(q1) with q0 = gate_qubits[2g].
 * gate_layer is informational and may be NULL.  All arrays are host memory
 * owned by the caller and are copied; they may be freed after the call. */
typedef struct tn_circuit {
    int32_t        n_qubits;
    int32_t        n_gates;
    const int32_t* gate_qubits;     /* [n_gates][2] */
    const double*  gate_matrices;   /* interleaved complex128, see above */
    const int32_t* gate_layer;      /* [n_gates] or NULL */
} tn_circuit;

typedef struct tn_network_s tn_network_t;
typedef struct tn_plan_s    tn_plan_t;

/* Circuit -> tensor network (SI, TN section, figure S2): one tensor per gate,
 * legs labelled by wires (q, t).  Host only.  Fails with TN_ERR_ARG on a qubit
 * index out of range, a gate acting twice on one qubit, n_qubits outside
 * [1, 64] or a NULL pointer.  The network is owned by the caller and freed
 * with tn_network_destroy(). */
tn_status tn_network_from_circuit(const tn_circuit* circuit, tn_network_t** out);

/* Number of wires carrying label (q, t) for t = 0..count-1: writes, for every
 * qubit q, the number of gates on q into gates_per_qubit[q] (so that the
 * output wire of q is (q, gates_per_qubit[q])).  Host only. */
tn_status tn_network_wire_counts(const tn_network_t* net, int32_t* gates_per_qubit, int32_t cap);

void tn_network_destroy(tn_network_t* net);

/* ---------------------------------------------------------------- plan */

#define TN_PREC_FP32    0  /* complex64 SIMT FMA (the plain FP32 path) */
#define TN_PREC_TF32    1  /* tcgen05 kind::tf32, FP32 accumulate */
#define TN_PREC_BF16X3  2  /* tcgen05 kind::f16, bf16 hi+lo split operands, FP32 accumulate */
#define TN_PREC_FP16X3  3  /* tcgen05 kind::f16, fp16 hi+lo split operands, FP32 accumulate;
                              every operand is scaled by a power of two that maps its largest
                              component into [2^14, 2^15) before the split, and the product is
                              scaled back exactly.  A plan records each intermediate's largest
                              component in its producer's epilogue; tn_contract_pair finds A's
                              and B's by one extra read of each */

typedef struct tn_plan_opts {
    uint64_t open_mask;              /* qubits left open: 2^popcount amplitudes per batch */
    int32_t  max_log2_intermediate;  /* bound on every per-slice intermediate (elements) */
    int32_t  min_log2_slices;        /* slice at least this many wires (0: only what the bound needs) */
    uint64_t seed;                   /* seeds the randomised order search */
    int32_t  trials;                 /* order-search trials (<= 0: default) */
    int32_t  precision;              /* TN_PREC_* */
    int32_t  complex_mult;           /* 4 (4M: Re = ArBr - AiBi, Im = ArBi + AiBr) or 3 (3M:
                                        T1 = ArBr, T2 = AiBi, T3 = (Ar+Ai)(Br+Bi) with the sums
                                        formed in FP32; Re = T1 - T2, Im = T3 - T1 - T2) for the
                                        tensor-core kernels; 3 with TN_PREC_FP32 gives
                                        TN_ERR_UNSUPPORTED (the CUDA-core path is 4M only; it
                                        also serves the tiny steps of TF32/BF16X3 plans) */
    int32_t  log2_batch_slices;      /* slices contracted together per chunk (<= 0: auto) */
    int64_t  max_arena_bytes;        /* device arena cap for one chunk (<= 0: 96 GiB) */
    int32_t  n_forced_slices;        /* wires the caller slices (0: the planner chooses them all) */
    const int32_t* forced_slice_qubit;  /* [n_forced_slices]: wire (qubit, t) of slice bit j, host */
    const int32_t* forced_slice_t;      /* internal wires only: 1 <= t < gates on that qubit */
    double   mem_weight;             /* order-search cost = MACs + mem_weight * elements moved
                                        (<= 0: 32) */
    int32_t  sm_pairs;               /* 1: tensor-core steps of 4M products with at least two
                                        full 128-row m tiles may run on SM pairs (cta_group::2:
                                        two SMs share each MMA of 256 rows, each holding its
                                        128 rows of A and half of B'); 0: one SM per tile.
                                        Results agree within the precision's rounding either
                                        way (the FP32 summation order of an MMA may differ).
                                        An implementation choice: the paper's processors have
                                        no counterpart.  Other values: TN_ERR_ARG */
} tn_plan_opts;

/* Fill opts with defaults: no open qubits, bound 2^30, no forced slices, seed 1,
 * 64 trials, FP32, 4M, automatic batch, 96 GiB arena, SM pairs on.  Index permutations are
 * always folded into the contraction's operand loads and result stores (SI,
 * figure S7a): there is no separate permute pass on the plan path.
 * Forced slices: the given wires take slice bits 0..n_forced_slices-1 (in the
 * given order) and the planner orders the rest of the network around them,
 * adding further slices only if the bound needs them; chunks then hold one
 * slice each.  TN_ERR_ARG for a wire that is not an internal wire. */
tn_status tn_plan_default_opts(tn_plan_opts* opts);

/* Find a contraction order and a slice set (SI, TN section: pairwise order as
 * a list of two-tuples; main text, section II: slicing under a bound on the
 * largest intermediate).  Host only; no CUDA call is made.  The network is
 * simplified first (SI, TN section: rank-1 and rank-2 tensors are absorbed into
 * neighbours; two tensors are pre-contracted when the result's rank is not
 * larger than the larger input's).  The plan keeps its own copy of the
 * network's data and is freed with tn_plan_destroy().  TN_ERR_PLAN if the open
 * qubits alone exceed the bound. */
tn_status tn_plan(const tn_network_t* net, const tn_plan_opts* opts, tn_plan_t** out);

typedef struct tn_plan_stats {
    int32_t  n_qubits;
    int32_t  n_open;                 /* k: 2^k amplitudes per batch */
    int32_t  n_leaves;               /* tensors after simplification */
    int32_t  n_steps;                /* pairwise contractions per slice */
    int32_t  log2_slices;            /* S */
    int32_t  log2_batch_slices;      /* slices per chunk = 2^this */
    int32_t  log2_max_intermediate;  /* largest per-slice intermediate */
    int32_t  precision;
    double   flops_per_slice;        /* 8 real flops per complex multiply-add */
    double   bytes_per_slice;        /* 8 B per complex64 element: operands read once, result written once */
    double   flops_per_chunk;        /* with slice-invariant parts shared inside a chunk */
    double   bytes_per_chunk;
    int64_t  arena_bytes;            /* device arena of one chunk */
    int32_t  k_histogram[40];        /* steps per log2(contracted size k), as figure S4 */
    int32_t  complex_mult;
    int32_t  n_kernel_launches_per_chunk;  /* before kernels are chosen: slice-dependent steps + 4
                                              (tn_plan_chunk_launches gives the exact count) */
} tn_plan_stats;

/* Sizes and work of a plan (host only): the per-slice and per-chunk flop and
 * byte counts behind the complexity figures of SI Table 1 (counted as 8 real
 * flops per complex multiply-add) and the histogram of contracted sizes k of
 * SI figure S4.  TN_ERR_ARG on a NULL argument. */
tn_status tn_plan_info(const tn_plan_t* plan, tn_plan_stats* out);

/* The sliced wires in slice-bit order: qubit[j], t[j] label slice bit j.
 * `count` receives S; at most `cap` entries are written. */
tn_status tn_plan_sliced_wires(const tn_plan_t* plan, int32_t* qubit, int32_t* t,
                               int32_t cap, int32_t* count);

/* Per-step shapes (for sweeps and reports): log2 of m (rows of the streamed
 * operand), k (contracted size), n (columns of the small operand) and of the
 * number of batch instances per chunk, for step i < n_steps. */
tn_status tn_plan_step_shape(const tn_plan_t* plan, int32_t step, int32_t* log2_m,
                             int32_t* log2_k, int32_t* log2_n, int32_t* log2_batch);

/* Storage layout of step i's operands (host only; no paper counterpart: an
 * introspection call for reports and tests).  Positions are bit positions of
 * each operand's element index (element = complex64, position 0 the fastest).
 * Writes to out[0..] in this order: nm, nk, nn, nb, then a_m[nm], a_k[nk],
 * b_k[nk], b_n[nn], c_m[nm], c_n[nn], a_b[nb], b_b[nb], c_b[nb], then the
 * step's dependence flags (bit 0: its result depends on the slice id, bit 1:
 * on the closed output bits; 0 = the same tensor in every chunk), then its
 * group id (steps sharing an id >= 0 are consecutive, independent, and none
 * writes where another of the group reads, so they run concurrently; -1: the
 * step runs alone): where A is
 * the streamed operand, B the small one, C the result, and a_m[j] / c_m[j] the
 * positions of row bit j in A and in C (and so on).  `count` receives the
 * number of entries; at most `cap` are written (TN_ERR_ARG if cap is too small). */
tn_status tn_plan_step_layout(const tn_plan_t* plan, int32_t step, int32_t* out, int32_t cap,
                              int32_t* count);

/* The plan's contraction tree in terms of the circuit (host only; the SI's
 * pairwise order as a list of two-tuples, over the simplified network): after
 * simplification every circuit gate belongs to exactly one leaf tensor, and
 * leaf_of_gate[g] (HOST [n_gates], n_gates >= the circuit's gate count)
 * receives that leaf's index in [0, n_leaves); step_nodes (HOST [2 cap_steps])
 * receives, for every step j in execution order, the two node ids it
 * contracts (leaves 0..n_leaves-1; the result of step j is node n_leaves + j).
 * The initial-state and output-projector tensors belong to the leaves that hold
 * their qubit's first and last gate.  For reports and for checking a plan's
 * partial sums against an independent contraction along the same tree.
 * TN_ERR_ARG when n_gates or cap_steps is too small. */
tn_status tn_plan_tree(const tn_plan_t* plan, int32_t* leaf_of_gate, int32_t n_gates, int32_t* step_nodes,
                       int32_t cap_steps, int32_t* n_leaves, int32_t* n_steps);

/* Modeled device time of one chunk of the plan on a roofline (host only; the
 * cost model of plan selection, SI: the order with the fewest flops is not the
 * fastest, so orders are compared by time): the sum over the steps that run in
 * every chunk (those whose result depends on the slice id; the others run
 * once per plan or per batch) of
 *     max(8 m k n / peak_flops, 8 (|A| + |B| + |C|) / peak_bytes)
 * with m, k, n the step's complex GEMM extents summed over its batch instances
 * and |A|, |B|, |C| its operands' complex64 element counts.  peak_flops in
 * algorithmic flop/s (8 per complex multiply-add) of the plan's precision,
 * peak_bytes in B/s, both > 0.  Writes seconds to *seconds. */
tn_status tn_plan_model_time(const tn_plan_t* plan, double peak_flops, double peak_bytes, double* seconds);

/* Contract slices [slice_first, slice_first + slice_count) for n_batches
 * correlated batches and ADD the result into out_amplitudes (main text, section
 * II: the sliced network is the sum of the slices; section III: one run gives
 * the 2^k amplitudes of a batch).
 *   open_bitstrings  host array [n_batches]: the closed bits of each batch
 *                    (bits at open positions ignored); copied before return.
 *   out_amplitudes   DEVICE array of n_batches * 2^k interleaved complex128,
 *                    accumulated (+=) in FP64; owned by the caller.
 *   stream           cudaStream_t; the call is asynchronous on it.
 * The first call on a plan allocates the plan's device arena, workspace and
 * the B' image buffers of steps whose B operand depends on no slice (all freed
 * by tn_plan_destroy) and uploads the leaf tensors; that call synchronises.
 * Steps that depend on no slice, and those B' images, are computed once per
 * plan, or once per batch when they depend on the closed bits (main text,
 * section III: the major part of the network is shared by a correlated batch).
 * A range beyond 2^S, n_batches < 1 or a NULL pointer gives TN_ERR_ARG.  Not
 * thread-safe per plan. */
tn_status tn_contract_slices(tn_plan_t* plan, uint64_t slice_first, uint64_t slice_count,
                             const uint64_t* open_bitstrings, int32_t n_batches,
                             double* out_amplitudes, void* stream);

/* Device time of every step's kernel: after the plan's device state exists
 * (one tn_contract_slices call), launches each step's GEMM `reps` times on
 * `stream` between CUDA events, on the arena contents of the last chunk, and
 * writes the mean milliseconds per launch into ms_out[n_steps] (host array)
 * and, when kernel_out is not NULL, the kernel used by each step into
 * kernel_out[n_steps]: 0-2 FP32 SIMT tiles (64x64, 128x16, 256x4), then the
 * tcgen05 kernels 3 TF32 4M, 4 BF16x3 4M, 5 TF32 3M, 6 BF16x3 3M, 7 FP16x3 4M,
 * 8 FP16x3 3M.  Used for plan reports and roofline measurements; synchronises
 * `stream`. */
tn_status tn_plan_step_times(tn_plan_t* plan, int32_t reps, double* ms_out, int32_t* kernel_out,
                             void* stream);

/* Autotuner (after one tn_contract_slices call): times candidate kernels for
 * every step in place on `stream` -- tensor-core tiles of 32, 64 or 128
 * complex columns in the TF32 / BF16X3 / FP16X3 modes, each with either
 * write-back order, with the default or a deeper ring of B' slots and, where
 * tn_plan_opts.sm_pairs allows, on one SM or on SM pairs, and the
 * three CUDA-core tilings for steps under 50 us, of low arithmetic intensity
 * or in the FP32 mode -- each `reps` times, and keeps the fastest for later
 * calls.  Synchronises `stream`; the arena contents are
 * overwritten (the next call recomputes them). */
tn_status tn_plan_autotune(tn_plan_t* plan, int32_t reps, void* stream);

/* The kernel chosen for every step (after one tn_contract_slices call; the
 * autotuner's choices once tn_plan_autotune ran), TN_TUNING_INTS int32 per step
 * in plan order: kernel id (as in tn_plan_step_times), tile width as log2
 * complex columns (-1: the CUDA-core default), write-back order (0 direct, 1
 * staged in C's memory order), B' ring slots (0 for CUDA-core kernels), SM
 * pair (0 or 1).  `out` is a host array of `cap` int32; *n_out receives the
 * count written (n_steps * TN_TUNING_INTS); TN_ERR_ARG if cap is too small.
 * With tn_plan_set_tuning it carries a tuning from one process to another (a
 * profiled run, whose own timing the profiler distorts, then runs the kernels
 * an unprofiled autotuner chose).  Host only; no device work.  The paper has no
 * counterpart (an implementation's kernel choice). */
#define TN_TUNING_INTS 5
tn_status tn_plan_get_tuning(const tn_plan_t* plan, int32_t* out, int32_t cap, int32_t* n_out);

/* Apply a tuning from tn_plan_get_tuning of a plan with the same steps (the
 * same network and tn_plan_opts), after one tn_contract_slices call on this
 * plan: every step gets the given kernel as the autotuner would have built it.
 * n must be n_steps * TN_TUNING_INTS; an unknown kernel id, or a choice the
 * step cannot take (a tensor-core kernel for the FP32 mode, rings that do not
 * fit), gives TN_ERR_ARG and leaves the plan's kernels unchanged.  Launches
 * nothing; it may resize the plan's device workspace and image buffers (which
 * synchronises the device).  The next contract call captures the chunk graph
 * again and reruns the prologues. */
tn_status tn_plan_set_tuning(tn_plan_t* plan, const int32_t* in, int32_t n);

/* Plan selection by measured time (SI, TN section: the order whose measured
 * slice time is smallest is kept, not the one with the fewest flops).  Builds
 * n_candidates plans from *opts with seeds seed, seed+1, ... and memory weights
 * cycling through w, w/4, 4w (w = opts->mem_weight or 32), times chunks of
 * each on `stream` (after an untimed warm-up call with the same bitstring, the
 * fastest of three timed calls of one chunk), estimates the time for all 2^S
 * slices as chunk time x 2^(S-b), and returns the fastest plan in *out (its
 * device state is released; the first contract call re-creates it).
 * cand_seconds (HOST, [n_candidates], may be NULL) receives each estimate, -1
 * for a candidate that could not be built or run (e.g. its arena does not
 * fit).  Synchronises `stream`; TN_ERR_PLAN if no candidate ran.  Kernels are
 * not autotuned during the selection. */
tn_status tn_plan_select(const tn_network_t* net, const tn_plan_opts* opts, int32_t n_candidates,
                         uint64_t open_bitstring, void* stream, tn_plan_t** out, double* cand_seconds);

/* tn_plan_select over a caller-given candidate list: candidate i is *opts with
 * seed seeds[i] and memory weight mem_weights[i] (HOST arrays [n_candidates],
 * n_candidates in [1, 1024]); timing, estimate, result and errors as in
 * tn_plan_select.  With tn_plan_rank this is the two-stage selection of a plan
 * pool: rank many orders by modeled time on the host, measure the best few. */
tn_status tn_plan_select_list(const tn_network_t* net, const tn_plan_opts* opts, int32_t n_candidates,
                              const uint64_t* seeds, const double* mem_weights, uint64_t open_bitstring,
                              void* stream, tn_plan_t** out, double* cand_seconds);

/* Host-only ranking of a plan pool (SI, TN section: many candidate orders are
 * generated and compared by time, since the order with the fewest flops is not
 * the fastest).  Candidate i is *opts with seed seeds[i] and memory weight
 * mem_weights[i] (HOST arrays [n_candidates], n_candidates in [1, 100000]);
 * each is planned (tn_plan) and model_seconds[i] (HOST) receives its modeled
 * time for one batch over all 2^S slices -- tn_plan_model_time(peak_flops,
 * peak_bytes) of one chunk x 2^(S-b), plus the same roofline sum over the
 * steps that run once per batch bitstring (they depend on the closed output
 * bits but on no slice) -- or -1 when the candidate cannot be planned (e.g. no
 * batch fits the arena cap).  Steps that depend on neither run once per plan
 * and are not counted.  Plans are built one after another, each on all host
 * cores, and freed.  No CUDA call is made.  TN_ERR_PLAN if no candidate could
 * be planned; TN_ERR_ARG on NULL arrays or non-positive peaks. */
tn_status tn_plan_rank(const tn_network_t* net, const tn_plan_opts* opts, int32_t n_candidates,
                       const uint64_t* seeds, const double* mem_weights, double peak_flops, double peak_bytes,
                       double* model_seconds);

/* Kernels one chunk launches with the kernels chosen so far (after the first
 * tn_contract_slices call; TN_ERR_ARG before): leaf select, every
 * slice-dependent step's kernels (tensor-core steps: B' image + GEMM [+ split-K
 * reduction]; CUDA-core steps: one), the two slice-sum kernels and the chunk
 * advance.  Steps that depend on no slice run once per plan or per batch and
 * are not counted.  Host only. */
tn_status tn_plan_chunk_launches(const tn_plan_t* plan, int32_t* launches);

/* Kernels the per-batch prologue launches (after the first tn_contract_slices
 * call; TN_ERR_ARG before): the steps that depend on the closed output bits
 * but on no slice run once for every new batch bitstring (main text, section
 * III: the part of the network shared by a batch's slices is contracted once),
 * each with its kernels as in tn_plan_chunk_launches, after one leaf select;
 * 0 when the plan has no such step.  Host only. */
tn_status tn_plan_batch_launches(const tn_plan_t* plan, int32_t* launches);

/* Wait for the plan's work on `stream` and return its sticky device error, if any. */
tn_status tn_plan_sync(tn_plan_t* plan, void* stream);

void tn_plan_destroy(tn_plan_t* plan);

/* ---------------------------------------------------------------- frugal sampling */

/* Frugal rejection sampling from one batch of correlated amplitudes (main
 * text, section III: a 2^k-amplitude batch from one contraction, then frugal
 * sampling, gives one sample with probability close to 1).  Sample s walks its
 * n_draws draws: draw t proposes batch member candidates[s * n_draws + t] with
 * uniform uniforms[s * n_draws + t] in [0, 1); the first draw with
 *     u * m_bound < 2^n_qubits * |a|^2
 * (products rounded separately, FP64) is accepted, so an accepted member is
 * distributed as min(1, N p / M) over the batch.  The random numbers are the
 * caller's (draw candidates uniformly from the batch).
 *   amplitudes  DEVICE complex128 [count] (a batch of tn_contract_slices)
 *   candidates  DEVICE int64 [n_samples * n_draws], each in [0, count)
 *   uniforms    DEVICE double [n_samples * n_draws]
 *   first_out   HOST int64 [n_samples]: the accepted draw t of each sample, or
 *               -1 if none of its draws is accepted (the sample is
 *               candidates[s * n_draws + first_out[s]]).
 * Synchronises `stream`.  Empty inputs, m_bound <= 0 or a candidate outside
 * [0, count) give TN_ERR_ARG (candidates are checked on the device). */
tn_status tn_frugal_sample(const double* amplitudes, int64_t count, int32_t n_qubits, double m_bound,
                           const int64_t* candidates, const double* uniforms, int64_t n_draws,
                           int64_t n_samples, int64_t* first_out, void* stream);

/* ---------------------------------------------------------------- XEB */

/* Linear XEB (main text, Eq. (1): the mean of x = N p is 1 + F):
 * F = 2^n_qubits * mean_i |a_i|^2 - 1 over `count` DEVICE complex128 amplitudes,
 * summed in FP64 on the device.  Writes F to the HOST double *xeb_out.
 * Synchronises `stream`.  count < 1 gives TN_ERR_ARG. */
tn_status tn_xeb(const double* amplitudes, int64_t count, int32_t n_qubits, double* xeb_out,
                 void* stream);

/* ---------------------------------------------------------------- kernels */

/* Index permutation of `batch` complex64 tensors of rank `rank` (every index of
 * dimension 2, index 0 fastest): out index position p carries the input index
 * at position perm[p] (SI, Eq. (2): the permutation that makes contracted
 * indices one matrix dimension).  in/out are DEVICE interleaved complex64
 * arrays of batch * 2^rank elements, not overlapping.  rank in [0, 34]. */
tn_status tn_permute(const float* in, float* out, int32_t rank, const int32_t* perm,
                     int64_t batch, void* stream);

/* One pairwise contraction C = sum_shared A * B of two DEVICE complex64
 * tensors (SI, Eq. (2)), through the same kernels as a plan step.  Wires are
 * arbitrary int32 ids, listed in storage order (position 0 fastest); a wire in
 * both A and B is contracted; c_wires must be the remaining wires in any order.
 * `batch` independent instances are stored back to back in each array.
 * precision and complex_mult as in tn_plan_opts; tensor-core products run on
 * SM pairs wherever tn_plan_opts.sm_pairs = 1 would let them.  Asynchronous on
 * stream; a device-side error (a bounded wait of the tensor-core kernel that
 * ran out, leaving C incomplete) is reported by the next tn_device_sync(). */
tn_status tn_contract_pair(const float* a, const int32_t* a_wires, int32_t a_rank,
                           const float* b, const int32_t* b_wires, int32_t b_rank,
                           float* c, const int32_t* c_wires, int32_t c_rank,
                           int64_t batch, int32_t precision, int32_t complex_mult,
                           void* stream);

/* Self-test of the bounded device waits that every tensor-core kernel uses:
 * launches one thread that waits on an mbarrier nothing ever arrives on, with
 * a limit of wait_ms milliseconds (1..5000), and writes the device error word
 * after the kernel into *device_status: TN_ERR_TIMEOUT when the wait gave up as
 * designed.  The word is left set, exactly as a timed-out contraction leaves
 * it, so the next tn_device_sync() reports TN_ERR_TIMEOUT and clears it.  The
 * kernel returns normally and the context stays usable.  The paper has no
 * counterpart (failure handling of this implementation).  Synchronises
 * `stream`. */
tn_status tn_selftest_bounded_wait(int32_t wait_ms, int32_t* device_status, void* stream);

/* Wait for `stream`, then read and clear the current device's error word of
 * the calls without a plan (tn_contract_pair, tn_contract_pair_noalloc,
 * tn_selftest_bounded_wait): TN_OK when no kernel of theirs reported an error
 * since the last tn_device_sync, else the recorded status (TN_ERR_TIMEOUT: a
 * bounded wait ran out and that call's output is incomplete).  The paper has
 * no counterpart (failure handling of this implementation).  Allocates
 * nothing, so callers of tn_contract_pair_noalloc may use it. */
tn_status tn_device_sync(void* stream);

/* tn_contract_pair without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory -- programs whose device memory belongs to another allocator (a
 * framework's caching pool, a fixed budget handed out at start-up), and
 * real-time or embedded hosts that forbid allocation once they run, because
 * an allocation can block, fail or fragment at a time they do not control.
 * Arguments, layouts and results are those of tn_contract_pair (same kernels,
 * same split-K choice while the partial sums fit the array); the caller still
 * provides A, B and C.
 *   - Scratch (an error word, the FP16X3 operand maxima, the B' images of the
 *     tensor-core kernels and any split-K partial sums) comes from one static
 *     device array of 32 MiB compiled into the library; every GPU that loads
 *     the library holds it until the process exits.  A contraction whose
 *     scratch exceeds it even without split-K (tensor-core paths: about 16
 *     bytes per complex entry of B per batch instance, after padding k to 16
 *     and n to 8) fails with TN_ERR_ARG before anything is launched.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.  The
 *     first call on each device looks the array's device address up (with
 *     that device current); make that first call before any stream capture.
 *   - Every call shares the array, which keeps the previous call's contents;
 *     what must start at zero (the operand maxima) is cleared on the stream by
 *     each call.  The error word is zero at load, only ever set by a kernel
 *     that gives up a bounded wait, and read and cleared by tn_device_sync().
 *     Calls that overlap on the GPU (other streams, other threads) race on the
 *     array and must be serialised by the caller.
 * Asynchronous on stream. */
tn_status tn_contract_pair_noalloc(const float* a, const int32_t* a_wires, int32_t a_rank,
                                   const float* b, const int32_t* b_wires, int32_t b_rank,
                                   float* c, const int32_t* c_wires, int32_t c_rank,
                                   int64_t batch, int32_t precision, int32_t complex_mult,
                                   void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TN_GB300_H */
