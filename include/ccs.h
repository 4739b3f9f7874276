/*
 * ccs.h -- C ABI of the GB300 (sm_103a) Clifford circuit-cutting hot path.
 *
 * The method is Clifford-based circuit cutting ("Clifford-based Circuit
 * Cutting for Quantum Simulation", Smith, Perlin et al.): a near-Clifford
 * circuit is cut into Clifford and small non-Clifford fragments (Sec. V-A),
 * every fragment *variant* -- one choice of prepared state at each quantum
 * input and of measurement basis at each quantum output (Sec. V-B) -- is
 * simulated, Clifford ones by a stabilizer tableau and the others by an exact
 * statevector (Sec. V-B), and the distribution of the uncut circuit is
 * rebuilt by a contraction over the 4^k cut terms (Sec. III-B, Sec. V-C).
 *
 * Three calls carry the path:
 *   ccs_build_fragments  circuit(s) -> fragments + variant plan      (Sec. V-A)
 *   ccs_eval_variants    plan -> per-variant outcome data on the GPU (Sec. V-B)
 *   ccs_recombine        per-variant data -> marginal + <Z_S> values (Sec. V-C)
 *
 * Conventions (fixed by this interface; the paper leaves them open):
 *   - qubits start in |0>, outputs are measured in Z (Sec. V-B);
 *   - a cut {qubit, gate_index} splits the qubit's wire just before gate
 *     gate_index of the flat gate list; cuts are ordered by (gate_index, qubit);
 *   - a fragment's wires are the wire segments it owns, ordered by
 *     (qubit, segment); fragments are ordered by their first wire;
 *   - preparations 0..3 = |0>,|1>,|+>,|+i>; bases 0..2 = X,Y,Z;
 *   - variant id = mixed radix: quantum inputs first (radix 4, first input
 *     least significant), then quantum outputs (radix 3), both in cut order;
 *   - measured list A_f = the fragment's marginal wires (in the caller's
 *     marginal order) then its quantum-output wires (cut order); bit j of an
 *     outcome y is wire A_f[j];
 *   - bit j of a marginal index is the j-th qubit of the caller's marginal.
 *
 * Ownership: every pointer passed in belongs to the caller and is only read
 * during the call (host memory unless stated).  Plans, results and contexts
 * belong to the library and are released by their *_free / ccs_destroy.
 * Device memory is taken from the context's allocator (see ccs_allocator).
 *
 * Errors: every int-returning call returns CCS_OK (0) or a negative
 * CCS_ERR_* code and leaves a message in ccs_last_error(ctx).  No exception
 * crosses the ABI.  A context must be used by one host thread at a time.
 * A plan may be evaluated and recombined by any context on the same device
 * (for example one thread building plans with its own context while another
 * evaluates them); the context that built a plan must outlive it, and a plan
 * or result is used by one thread at a time.
 */
#ifndef CCS_ABI_H_
#define CCS_ABI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CCS_OK 0
#define CCS_ERR_INVALID_ARG (-1)
#define CCS_ERR_UNSUPPORTED_GATE (-2)
#define CCS_ERR_TOO_MANY_CUTS (-3)
#define CCS_ERR_NC_TOO_WIDE (-4)
#define CCS_ERR_OOM (-5)
#define CCS_ERR_CUDA (-6)
#define CCS_ERR_TIMEOUT (-7)
#define CCS_ERR_UNSUPPORTED (-8)
#define CCS_ERR_DEVICE_CHECK (-9)

/* Gate opcodes (Sec. II-A, II-C): Paulis, S = Z^{1/2}, H, CX, CZ; T = Z^{1/4}
 * and its inverse are the non-Clifford gates.  CCS_ZPOW is Z^a =
 * diag(1, e^{i pi a}) with a = param (Sec. VIII: the cutter isolates any Z^a):
 * when 2a is an integer it is the Clifford S^{2a} (identity, S, Z or S^dagger)
 * and is simulated as such; otherwise it is non-Clifford and its wire segment
 * goes to a statevector fragment like a T gate. */
enum {
  CCS_H = 0, CCS_S = 1, CCS_SDG = 2, CCS_X = 3, CCS_Y = 4, CCS_Z = 5,
  CCS_CX = 6, CCS_CZ = 7, CCS_T = 8, CCS_TDG = 9, CCS_ZPOW = 10
};

/* One gate.  q[1] is the target of CX (q[0] the control) and is ignored for
 * one-qubit gates.  param is the exponent a of CCS_ZPOW (finite, else
 * CCS_ERR_INVALID_ARG) and ignored for the other opcodes; nq and flags are
 * reserved (set to 0). */
typedef struct {
  uint8_t op;
  uint8_t nq;
  uint16_t flags;
  uint32_t q[2];
  double param;
} ccs_gate;

typedef struct {
  uint32_t qubit;
  uint32_t gate_index;
} ccs_cut;

/* One problem: a circuit, its cuts and what to report.
 *   cuts/n_cuts   explicit wire cuts; n_cuts < 0 asks ccs_build_fragments to
 *                 search for a cut set (greedy, or the learned scorer);
 *   marginal      output qubits of the reported marginal (<= 24 of them);
 *   zstring_*     CSR list of Z-strings S (sets of qubits): <Z_S> is
 *                 reported for each. */
typedef struct {
  uint32_t n_qubits;
  uint32_t n_gates;
  const ccs_gate* gates;
  int32_t n_cuts;
  const ccs_cut* cuts;
  uint32_t n_marginal;
  const uint32_t* marginal;
  uint32_t n_zstrings;
  const uint32_t* zstring_offsets;   /* n_zstrings + 1 entries */
  const uint32_t* zstring_qubits;
} ccs_problem;

typedef struct ccs_ctx_s* ccs_ctx;
typedef struct ccs_plan_s* ccs_plan;
typedef struct ccs_res_s* ccs_res;

/* Device allocator: alloc returns device memory of `bytes` usable on
 * `stream` (NULL on failure); free releases it.  Passing NULL to ccs_create
 * uses cudaMallocAsync / cudaFreeAsync on the context's stream. */
typedef void* (*ccs_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*ccs_free_fn)(void* ptr, size_t bytes, void* stream, void* user);
typedef struct {
  ccs_alloc_fn alloc;
  ccs_free_fn free;
  void* user;
} ccs_allocator;

/* Create a context on CUDA device `device`, issuing all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * device < 0 creates a host-only context: plans can be built and inspected
 * (fragments, cuts, variant counts) without a GPU; ccs_eval_variants and
 * ccs_recombine then return CCS_ERR_UNSUPPORTED.  Without an allocator the
 * context takes device memory from a stream-ordered pool the library keeps
 * per device (shared by all such contexts): freed memory stays in the pool
 * for the next plan or result, and ccs_destroy hands the unused part back
 * to the driver. */
int ccs_create(ccs_ctx* out, int device, void* cuda_stream, const ccs_allocator* alloc);
void ccs_destroy(ccs_ctx ctx);
const char* ccs_last_error(ccs_ctx ctx);
/* Library version string (static storage). */
const char* ccs_version(void);
/* Kernels the library has launched in this process so far (a replayed CUDA
 * graph adds its kernel nodes once per replay).  Diagnostic, no counterpart
 * in the paper; never fails. */
long long ccs_launch_count(void);

/* --- cutting (Sec. V-A) --------------------------------------------------- */
typedef struct {
  int32_t max_cuts;        /* reject / bound searched cut sets (default 12) */
  int32_t max_nc_width;    /* widest non-Clifford fragment allowed (<= 12) */
  int32_t use_learned;     /* 1: let the learned scorer pick among candidates */
} ccs_cut_opts;

/* Split each problem's circuit at its cuts into fragments, build every
 * fragment's variant list, compile its gates into moments of fused one- and
 * two-qubit Clifford updates (Clifford fragments) or 2x2 / 4x4 unitaries
 * (non-Clifford fragments), and upload the plan to the device.
 * Errors: INVALID_ARG (bad qubit index, cut position, marginal, Z^a
 * exponent; an empty circuit; more than 2^24 qubits or 2^30 gates),
 * UNSUPPORTED_GATE, TOO_MANY_CUTS, NC_TOO_WIDE, UNSUPPORTED (a cut whose two
 * ends lie in the same fragment; a Clifford fragment wider than 1024 wires;
 * a fragment measuring more than 24 wires; more than 13 fragments in one
 * problem), OOM (device, or a failed host allocation), CUDA.  Plans may be
 * built on several host threads at once, each with its own context; the
 * build uses the library's host worker pool and waits only for its own
 * upload, not for other work on the context's stream. */
int ccs_build_fragments(ccs_ctx ctx, const ccs_problem* problems, int n_problems,
                        const ccs_cut_opts* opts, ccs_plan* out);
/* Free a plan.  Its device memory goes back to the allocator of the context
 * that built it, on that context's stream (stream-ordered with the default
 * allocator): work that reads the plan on other streams must be complete
 * first. */
void ccs_plan_free(ccs_plan plan);

/* Candidate cut sets of one problem from the cut search (its cuts field is
 * ignored), cheapest first by the search's work estimate: a greedy beam over
 * regions grown from the non-Clifford gates (Sec. V-A: cuts isolate the
 * non-Clifford operations).  Candidate i's cuts are
 * cuts_out[offsets[i] .. offsets[i+1]) in cut order, its estimate costs[i].
 * Returns the number of candidates written (<= cap_cands; offsets needs
 * cap_cands + 1 entries) or an error (TOO_MANY_CUTS when no candidate fits
 * the limits).  Works on host-only contexts. */
int ccs_cut_candidates(ccs_ctx ctx, const ccs_problem* problem, const ccs_cut_opts* opts,
                       ccs_cut* cuts_out, int cap_cuts, int* offsets, double* costs, int cap_cands);

/* --- variant evaluation (Sec. V-B) ---------------------------------------- */
#define CCS_EXACT 0
#define CCS_SAMPLED 1
/* Clifford-specific stitching (Sec. IX): every Pauli expectation of a
 * stabilizer state is -1, 0 or +1 and follows from the state without
 * shots, and the Pauli terms that vanish contribute nothing downstream.
 * In this mode every Clifford variant is exact (as CCS_EXACT); a star
 * hub's contraction operand (one row per preparation tuple and output
 * Pauli string) is formed in closed form from each variant's outcome space
 * -- a row is either identically zero, when its sign mask is not
 * orthogonal to the space's purely quantum-output directions, or +-2^-r
 * times a sign affine in the outputs on the space's projection -- without
 * shots or per-variant distributions, and the contraction skips the rows
 * that vanish.  Results equal CCS_EXACT's up to FP32 rounding order. */
#define CCS_STITCH 2
typedef struct {
  int32_t mode;            /* CCS_EXACT: closed-form 2^-rank per Clifford variant;
                              CCS_SAMPLED: `shots` Philox shots per Clifford variant;
                              CCS_STITCH: CCS_EXACT with the hub operand in closed form
                              and its vanishing rows skipped */
  uint32_t shots;
  uint32_t seed_lo, seed_hi;   /* Philox4x32-10 key */
  int32_t keep_tableaus;   /* 1: keep every final tableau (ccs_get_tableau) and the
                              star hub's dense shot counts (ccs_get_counts) */
  int32_t use_graph;       /* 1: capture the launches in a CUDA graph and replay */
  int32_t autotune;        /* 1: before the first launch of this result, time the
                              candidate launch shapes on this plan and keep the
                              fastest (cached in the context per shape bucket) */
  int32_t per_variant_body; /* 1: simulate each variant's whole gate sequence; 0 (default):
                              evolve each Clifford fragment's shared body once and derive
                              every variant from it (same tableaus bit for bit) */
  int32_t hub_sampler;     /* star hubs' sampler: 0 automatic (or autotuned), 1 16-bit
                              counters, 2 byte counters with an exact 16-bit recount where
                              a byte could overflow, 256 threads per CTA, 3 the same with 512
                              (2 and 3 used only if every hub has >= 2 marginal bits, <= 4
                              quantum outputs, |A| <= 16); same counts */
} ccs_eval_opts;

/* Evaluate every variant of every fragment of the plan on the GPU: tableau
 * evolution, GF(2) reduction to the affine outcome space, Philox sampling
 * (Clifford) or complex64 statevectors (non-Clifford), then the fold of the
 * variant data into one tensor per fragment.  By default each Clifford
 * fragment's gates are evolved once (the body) and every variant's outcome
 * space and Z-string values follow from the body without a tableau per
 * variant; with keep_tableaus each variant's final tableau is formed too
 * (same results bit for bit).  Philox call (g, v, f, c) (counter words:
 * call index, variant, fragment, problem) yields four 32-bit words of the
 * variant's stream; shot t takes field t mod s of word t div s, s = 4 / 2 / 1
 * shots per word when the space's rank is <= 8 / <= 16 / above, and uses the
 * field's low rank bits.  If *res is NULL a result is created, else its
 * buffers are reused (same plan only).  The call is asynchronous on the
 * context stream; getters synchronise. */
int ccs_eval_variants(ccs_ctx ctx, ccs_plan plan, const ccs_eval_opts* opts, ccs_res* res);
/* Free a result (its device memory goes back on the context's stream). */
void ccs_res_free(ccs_res res);
/* Launch shape in use for a result (after autotuning, if any): threads per
 * tableau CTA, 64-row words of one fused op per thread, shots per sampling
 * CTA, threads per fused hub-sampler CTA (negative: the byte-counter
 * sampler with that many threads), and the evaluation path (1: every
 * Clifford variant simulates its whole circuit, which the autotuner picks
 * for small plans when it is faster, or which per_variant_body asks for;
 * 0: shared bodies and the outcome-space screen).  Both paths give the same
 * outcome spaces, shots and values.  Any output may be NULL. */
int ccs_get_tuning(ccs_ctx ctx, ccs_res res, int* cliff_threads, int* words_per_op, int* shots_per_cta,
                   int* hub_threads, int* variant_path);

/* --- recombination (Sec. V-C) --------------------------------------------- */
#define CCS_FP32 0
#define CCS_BF16 1
typedef struct {
  int32_t precision;          /* CCS_FP32 or CCS_BF16 operands of the 4^k contraction */
  int32_t outputs_on_device;  /* 1: marginal_out / zexp_out are device pointers */
  int32_t no_tensor_cores;    /* 1: BF16 contractions on CUDA cores even where the
                                 tcgen05 GEMM applies (0: use it, the default) */
  int32_t use_graph;          /* 1: capture the contraction launches in a CUDA graph
                                 kept on the result (per precision and tensor-core
                                 choice) and replay it (full cut-index range only) */
  uint64_t k_lo, k_hi;        /* sum only the cut-index terms P in [k_lo, k_hi) of every
                                 problem (clamped to its 4^k; k_hi = 0: to the end).
                                 Partial results over disjoint ranges add up to the
                                 full one: the split a multi-GPU contraction reduces
                                 with one FP64 sum.  Partial ranges run on CUDA cores. */
} ccs_recomb_opts;

/* p(o) = 2^-k sum_{P in {I,X,Y,Z}^k} prod_f T_f(o_f, P|f) for every problem
 * (Sec. V-C: one tensor per fragment, one index per cut), written to
 * marginal_out (problems back to back, 2^n_marginal doubles each) and <Z_S>
 * to zexp_out (n_zstrings doubles each).  Any fragment topology: a star (one
 * fragment on every cut) is contracted leaf by leaf or as a GEMM over the cut
 * index; chains and trees are summed over the whole cut index per output.
 * Partial sums over the cut index are combined in FP64.  Synchronises the
 * context stream unless outputs_on_device is set.  Errors: INVALID_ARG,
 * CUDA. */
int ccs_recombine(ccs_ctx ctx, ccs_plan plan, ccs_res res, const ccs_recomb_opts* opts,
                  double* marginal_out, double* zexp_out);

/* Recombination that allocates no device memory.  The paper has no
 * counterpart; this exists for callers that cannot allocate at the point
 * where they need the result: for example a runtime that reserved the whole
 * device for its own memory pool up front, or a latency-critical thread that
 * must not take the allocator's locks or risk the device-wide
 * synchronisation a cudaMalloc can cause.
 *
 * Same result as ccs_recombine (same kernels, same arithmetic), written
 * straight to the caller's DEVICE buffers marginal_out and zexp_out (layouts
 * as in ccs_recombine); the call is asynchronous on the context stream and
 * does not synchronise.  Its scratch (the leaves' Kronecker operand and the
 * split-K partials) is a fixed 8 MiB array inside the library that every
 * GPU loading the library holds until exit; a plan needing more
 * (4 * sum over problems of (4^k * N + splits * M * N) bytes) is rejected
 * with CCS_ERR_UNSUPPORTED.  Every scratch word is written before it is read
 * within one call, so nothing needs clearing, but all calls share the one
 * array: calls that may overlap on the GPU (other streams, other contexts
 * on the same device) race and must be ordered by the caller.  The first
 * call on each device looks up the array's device address; make that first
 * call before any stream capture.  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
int ccs_recombine_noalloc(ccs_ctx ctx, ccs_plan plan, ccs_res res, int precision, double* marginal_out,
                          double* zexp_out);

/* --- maximum-likelihood correction of fragment models (Sec. V-C) ----------- */
#define CCS_ML_SAMPLED 0   /* the fragments estimated from shots: the Clifford fragments of a
                              CCS_SAMPLED result (nothing to do for an exact result) */
#define CCS_ML_ALL 1       /* every fragment; exactly evaluated ones are physical already and
                              come back unchanged up to FP32 rounding */
/* Before the contraction, turn the selected fragments' data into physical
 * (self-consistent) fragment models, in place on the result (Sec. V-C:
 * maximum-likelihood corrections that mitigate sampling error).  The
 * paper names the step and its purpose only; the reading implemented:
 * fragment f's model is its Choi form, one operator per outcome o of its
 * marginal wires on its d cut slots (slot order),
 *   J_o = 2^-d sum_P T_f(o, P) (x)_j s_j(P_j),
 * s_j(P) = P^T where slot j is a quantum input and P where it is a quantum
 * output; physical means every J_o positive semidefinite with
 * sum_o Tr J_o = 2^{q_in}; the maximum-likelihood model under Gaussian shot
 * noise of equal variance per T_f entry is the physical model nearest in
 * Frobenius norm: all blocks' eigenvalues are projected together onto
 * {lambda >= 0, sum = 2^{q_in}} and each block is rebuilt from its own
 * eigenvectors (Smolin, Gambetta and Smith, PRL 108, 070502, 2012).  The
 * Z-string values are exact in every mode and are left alone.
 *
 * Afterwards ccs_recombine contracts the corrected models, ccs_get_tensor
 * returns them (hubs included) and ccs_get_operand the corrected operands
 * (FP32); the next ccs_eval_variants replaces them with raw data again.
 * Eigendecompositions run in complex64 (cyclic Jacobi), one CTA per block.
 * Asynchronous on the context stream.  Errors: INVALID_ARG (bad arguments,
 * a CCS_STITCH result), UNSUPPORTED (a selected fragment with more than 6
 * cut slots; a host-only context), OOM (its scratch: 4 D + 8 D^2 bytes per
 * block, D = 2^d), CUDA. */
int ccs_ml_correct(ccs_ctx ctx, ccs_plan plan, ccs_res res, int which);

/* --- learned cut scorer ------------------------------------------------------ */
/* A message-passing network over a circuit's qubit interaction graph with a
 * candidate cut set applied predicts log(evaluation + recombination time);
 * ccs_build_fragments with use_learned = 1 scores the cut search's
 * candidates with the context's model and takes the fastest predicted one,
 * unless the search's own estimate rates it more than 16x worse than its
 * best (then, and without a model, the greedy choice stands).  Fixed shape:
 * 8 node features, 8 global features, 3 layers of width 64; weights are
 * FP16 copies of an FP32 master; every step runs in the library's kernels.
 * Layout of the flat parameter vector: W_in (64x8), b_in, then per layer
 * W_self (64x64), W_neigh (64x64), b, then W_r1 (64x72), b_r1, w_r2 (64),
 * b_r2. */
typedef struct ccs_mpnn_s* ccs_mpnn;
/* A batch of graphs, host arrays: node features x (n_nodes x 8), CSR of the
 * normalised adjacency A (rowptr n_nodes+1, col, val) and the values of A^T
 * on the same pattern (val_t), graph_off (n_graphs+1) delimiting each
 * graph's nodes, glob (n_graphs x 8). */
typedef struct {
  int32_t n_nodes, n_graphs;
  const float* x;
  const int32_t* rowptr;
  const int32_t* col;
  const float* val;
  const float* val_t;
  const int32_t* graph_off;
  const float* glob;
} ccs_graph_batch;

int ccs_mpnn_num_params(void);
int ccs_mpnn_create(ccs_ctx ctx, uint64_t seed, ccs_mpnn* out);
void ccs_mpnn_free(ccs_mpnn net);
int ccs_mpnn_params(ccs_ctx ctx, ccs_mpnn net, float* out);          /* FP32 master copy */
int ccs_mpnn_set_params(ccs_ctx ctx, ccs_mpnn net, const float* in);
/* Predicted log times, one per graph (host output). */
int ccs_mpnn_forward(ccs_ctx ctx, ccs_mpnn net, const ccs_graph_batch* batch, float* pred);
/* Mean squared error against target and its gradient w.r.t. the parameters. */
int ccs_mpnn_gradient(ccs_ctx ctx, ccs_mpnn net, const ccs_graph_batch* batch, const float* target, float* loss,
                      float* grad);
/* One Adam step (beta 0.9, 0.999) on the mean squared error. */
int ccs_mpnn_train_step(ccs_ctx ctx, ccs_mpnn net, const ccs_graph_batch* batch, const float* target, float lr,
                        float* loss);
/* Node features (n_qubits x 8), CSR of A and A^T values (cap_nnz entries) and
 * the 8 global features of a problem under a cut set; returns nnz. */
int ccs_featurize(ccs_ctx ctx, const ccs_problem* problem, const ccs_cut* cuts, int n_cuts, float* x,
                  int32_t* rowptr, int32_t* col, float* val, float* val_t, int cap_nnz, float* glob);
/* Model used by ccs_build_fragments when use_learned is set (NULL: none). */
int ccs_set_cut_model(ccs_ctx ctx, ccs_mpnn net);

/* --- plan inspection -------------------------------------------------------- */
typedef struct {
  int32_t n_wires;
  int32_t clifford;
  int32_t n_variants;
  int32_t n_qin, n_qout;
  int32_t n_marg;           /* marginal bits owned by this fragment */
  int32_t n_meas;           /* |A_f| = n_marg + n_qout */
  int32_t n_slots;          /* cuts incident to the fragment */
  int32_t n_ops, n_moments; /* compiled gate stream */
  int32_t n_zstrings;       /* the problem's Z-strings (each restricted to the fragment) */
} ccs_fragment_info;

int ccs_plan_counts(ccs_ctx ctx, ccs_plan plan, int problem, int* n_fragments, int* n_cuts);
int ccs_fragment_info_get(ccs_ctx ctx, ccs_plan plan, int problem, int fragment,
                          ccs_fragment_info* out);
/* The cut set used for a problem (after search), in cut order. */
int ccs_plan_cuts(ccs_ctx ctx, ccs_plan plan, int problem, ccs_cut* out, int cap);
/* Wires of a fragment as (qubit, segment) pairs, 2*n_wires uint32. */
int ccs_fragment_wires(ccs_ctx ctx, ccs_plan plan, int problem, int fragment, uint32_t* out);

/* --- stage timing ------------------------------------------------------------ */
/* With profiling on, ccs_eval_variants runs without a CUDA graph and records
 * CUDA events on the context stream around each kernel stage; recombination
 * does the same.  ccs_get_stage_times synchronises the stream and writes the
 * last recorded duration of each stage in milliseconds (-1 if the stage did
 * not run) to ms[0..5]: 0 tableau evolution + outcome space + Z values
 * (one persistent kernel), 1 Philox sampling, 2 statevectors, 3 fold of the
 * Clifford fragments, 4 recombination, 5 contraction operands (the hub's
 * output-folded Q and the other fragments' preparation-weighted T').
 * Returns the number of stages (6) or an error; cap >= 6. */
int ccs_set_profiling(ccs_ctx ctx, int on);
int ccs_get_stage_times(ccs_ctx ctx, double* ms, int cap);

/* --- result getters (parity; caller-owned host buffers) ------------------ */
/* Final tableau of a Clifford variant (needs keep_tableaus): uint8
 * [2n][2n+1], row i = x_0..x_{n-1}, z_0..z_{n-1}, r; rows 0..n-1 are
 * destabilizers, n..2n-1 stabilizers. */
int ccs_get_tableau(ccs_ctx ctx, ccs_res res, int problem, int fragment, int variant, uint8_t* out);
/* Canonical affine outcome space of a Clifford variant: outcomes are
 * off ^ span(basis[0..rank)), basis in reduced row-echelon form with the
 * pivot (lowest set bit) ascending; off has every pivot bit clear. */
int ccs_get_outcome_space(ccs_ctx ctx, ccs_res res, int problem, int fragment, int variant,
                          uint64_t* off, uint64_t* basis, int* rank);
/* Shot counts of a sampled Clifford variant, 2^|A_f| uint32. */
int ccs_get_counts(ccs_ctx ctx, ccs_res res, int problem, int fragment, int variant, uint32_t* out);
/* Probabilities of a variant over 2^|A_f| outcomes (float32): exact ones for
 * non-Clifford variants, exact-mode Clifford variants and, in CCS_STITCH
 * mode, Clifford variants of fragments that are not a star's hub (a
 * stitched hub forms no per-variant distribution: INVALID_ARG). */
int ccs_get_dist(ccs_ctx ctx, ccs_res res, int problem, int fragment, int variant, float* out);
/* Z-string values of a variant (float32, nz x 2^n_qout, row-major): entry
 * [s][u] is <Z_S prod_{o in u} M_o> of the fragment's final state, S the
 * string's wires in the fragment, M_o the observable measured at quantum
 * output o (the cut identity, Sec. IV); +-1 or 0 for Clifford variants. */
int ccs_get_zvals(ccs_ctx ctx, ccs_res res, int problem, int fragment, int variant, float* out);
/* Contraction operand of a fragment of a star (float32, 2^n_marg x 4^n_slots):
 * for the hub Q[o][d] with d's digit at each cut = the preparation index where
 * the hub has a quantum input and the Pauli index where it has a quantum
 * output; for the other fragments T'[o][d] = T_f with the preparation weights
 * applied at the cuts where the fragment feeds the hub.  Then
 * p(o) = 2^-k sum_d Q[o_hub][d] prod T'[o_f][d|f]. */
int ccs_get_operand(ccs_ctx ctx, ccs_res res, int problem, int fragment, float* out);
/* Folded fragment tensor T_f[o][P] (float32, 2^n_marg x 4^n_slots, row-major).
 * For the hub of a star this is computed on request (the contraction uses
 * the hub's output-folded data directly). */
int ccs_get_tensor(ccs_ctx ctx, ccs_res res, int problem, int fragment, float* out);

#ifdef __cplusplus
}
#endif
#endif /* CCS_ABI_H_ */
