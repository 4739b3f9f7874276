// Device-side plan records and kernel launchers of the circuit-cutting hot path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "plan.hpp"

namespace ccs {

// One fragment as the kernels see it (all offsets index flat device arrays).
struct FragDev {
  int n, W, Wh;            // wires; tableau words per column (2*Wh) and per half
  int nA, m, qin, qout;    // |A_f|, marginal bits, quantum inputs / outputs
  int nv, clifford;        // variants; 1 = tableau, 0 = statevector
  int problem, findex;     // Philox counter words 3 and 2
  int ops_off, mom_off, n_moments;
  int A_off, qin_off, qout_off;   // into the wire-list array
  int nz, zw_off;          // Z-strings: nz+1 offsets at zoffs[zw_off..] into the wire-list array
  int n_slots;
  int slot_code[kMaxCuts]; // (kind << 8) | index into qin/qout
  int slot_cut[kMaxCuts];  // cut id within the problem
  int marg_pos[kMaxMarginal];
  long long space_off;     // SpaceRec index of variant 0
  long long counts_off;    // uint32 index of variant 0 (2^nA each)
  long long dist_off;      // float index of variant 0 (2^nA each)
  long long zval_off;      // float index of variant 0 (nz * 2^qout each)
  long long tab_off;       // uint64 index of variant 0 ((2n+3)*W each), -1 if not kept
  long long T_off;         // float index of T_f (2^m x 4^n_slots); also indexes TQ
  int role;                // 0 plain, 1 hub of a star (TQ = Q), 2 other fragment of a star (TQ = T')
  long long body_off;      // uint64 index of the shared body tableau ((2n+3)*W words), Clifford only
  long long rb_off;        // uint64 index of the fragment's kRowBasisWords (shared-row basis + offset table)
  long long zimg_off;      // uint64 index of the Z images (nz + 3 qout + m records of 2 Wh + 1 words)
  long long pb_off;        // uint32 index of the projected shared-row bases, 25 words per output basis
                           // combination (3^qout of them), -1 when qout > kMaxPbQout
  long long qrow_off;      // byte index of a Clifford hub's operand-row flags (4^n_slots), -1 otherwise
};

// Canonical affine outcome space of a Clifford variant.
struct SpaceRec {
  uint32_t off;
  int32_t rank;
  uint32_t basis[kMaxMeas];
  uint32_t flags;          // nonzero: a device-side consistency check failed
  uint32_t pad;
};

struct ProblemDev {
  int k, n_frags, frag0;   // cuts, fragments, first FragDev index
  int hub;                 // local index of the star's hub
  int n_marg, nz;
  long long marg_off, zexp_off;   // double indices into the outputs
  // contraction C[o_hub, o_leaf] = sum_P T_hub[o_hub, P] R[P, o_leaf] (star only)
  int M, N, splits;        // 2^m_hub, 2^(n_marg - m_hub), split-K factor
  int TM, TN, mtiles, ntiles;
  long long K;             // 4^k
  long long r_off;         // float index of R (K x N) in the scratch
  long long part_off;      // float index of the split-K partials (splits x M x N), after all R
  long long blk_off;       // first GEMM block of this problem
  long long rt_off;        // bf16 index of R'^T (N x K) in the bf16 scratch (tensor-core path)
  long long hub_T_off;     // T_off of the hub
  long long hub_qrow_off;  // qrow_off of the hub (-1: not a Clifford hub)
  int tc;                  // 1: eligible for the tensor-core GEMM in BF16 mode
  int direct;              // 1: contracted leaf by leaf in shared memory, TM hub outputs per CTA
  int general;             // 1: no fragment on every cut (not a star): every output summed over the
                           //    cut index from all fragment tensors (general_contract_kernel)
  int direct_staged;       // 1: the slice's hub operand (K x TM) is staged first; 0: the first leaf streams it
  // streaming CUDA-core GEMM of a wide hub (FP32, or BF16 off the tensor cores):
  // sthreads threads x 4 hub outputs per CTA, smblocks CTAs across M, ssplits across K
  int stream, sthreads, smblocks, ssplits;
  // the first leaf contracted while streaming (FP32, full range, dense rows):
  // its G1 = 4^s1 cut-digit rows per group against its table (N1 outputs),
  // then the other leaves' product table Rrest[group][NR] (NR = N / N1)
  int fact, fl1, G1, N1, NR;
  long long fl1_T_off;     // T_off of that leaf (its table T'[x1][g1])
  int ndig1, ndigr;
  int dig1[kMaxCuts], digr[kMaxCuts];   // cut positions of the leaf's digits / of the other digits
};

// Device views of a plan + result.
struct DevPlan {
  const FragDev* frags;
  const CliffordOp* cops;
  const NCOp* nops;
  const int* moments;
  const int* wires;
  const int* zoffs;
  const int2* items_cliff;    // (frag, variant), costliest first
  const int2* items_nc;       // (frag, first variant) of every statevector item
  int nc_basis_chunk;         // basis combinations an item covers (variants v0, v0 + 4^qin, ...)
  int n_items_cliff, n_items_nc;
  const int2* items_body;     // (frag, 64-row word) of every Clifford fragment's body
  int n_items_body, max_body_cols;
  int max_body_stage_words;   // body kernel shared memory with the op stream staged
  int max_moment_ops;         // widest gate moment of any Clifford fragment
  const int* cliff_frags;     // every Clifford fragment (shared-row bases)
  int n_cliff_frags;
  const int2* items_zimg;     // (frag, record) of every Z-image record
  int n_items_zimg;
  const int2* items_proj;     // (frag, output basis combination) of every projected shared-row basis
  int n_items_proj;
  const int2* zblocks;        // (frag, first variant) of each block of Z-string values
  int n_zblocks;
  int body_words_max;         // widest Clifford body tableau, uint64 words
  int img_words_max;          // most Z-image words of one fragment
  const ProblemDev* problems;
  int n_problems;
  const CliffordOp* prep_ops;  // 4
  const CliffordOp* basis_ops; // 3
  const float* prep_mats;      // 4 x 8
  const float* basis_mats;     // 3 x 8
};

struct DevRes {
  SpaceRec* spaces;
  uint32_t* counts;
  float* dist;
  float* zval;
  unsigned long long* tabs;
  unsigned long long* body;   // body tableaus, one per Clifford fragment
  unsigned long long* rowbasis;   // shared-row bases, 65 words per Clifford fragment
  unsigned long long* zimg;   // Z images: backward images of the Z-strings and measured Paulis
  unsigned* fragcnt;          // per Clifford fragment: measurement records done (zeroed per evaluation)
  uint32_t* pbasis;           // projected shared-row bases (pivot slots 0..23 + pivot mask)
  float* T;
  float* TQ;               // contraction operands: Q for hubs, T' for the other fragments
  uint16_t* TQh;           // bf16 copy of the hubs' Q (tensor-core path), may be null
  double* marg;
  double* zexp;
  uint8_t* qnz;            // stitched results: per Clifford hub operand row, 1 unless identically zero
  int hub_i16;             // sampled results (<= 32767 shots): the Clifford hubs' operands hold their
                           // signed count sums as int16 (value = sum x hub_scale), half the bytes
  float hub_scale;         // 1 / shots
  unsigned int* work;         // persistent-kernel work counters
  unsigned int* status;       // device-side error word
};

// Per Clifford fragment: the shared-row basis (64 pivot slots + pivot mask),
// the offset table of its measured Paulis (64 commutation-parity words + 64
// info words), and the extended vectors of each quantum input's body rows
// (kMaxCuts destabilizer words, then kMaxCuts stabilizer words).
constexpr int kRowBasisWords = 65 + 128 + 2 * kMaxCuts;
constexpr int kRbInputRows = 193;
// Fragments with at most this many quantum outputs get their shared-row
// basis projected once per output basis combination (3^qout <= 81).
constexpr int kMaxPbQout = 4;

// Largest intermediate (floats) of a star contracted leaf by leaf in shared
// memory; larger stars take the R / GEMM / reduce chain.
constexpr long long kDirectSmemFloats = 12288;

// Variants per block of Z-string values (about 256 (variant, string) pairs).
__host__ __device__ inline int zblock_variants(int nz) { return nz >= 256 ? 1 : 256 / nz; }

// Philox4x32-10 round keys of the key (seed_lo, seed_hi): round r uses
// (seed_lo + r W0, seed_hi + r W1) mod 2^32, W0 = 0x9E3779B9, W1 = 0xBB67AE85
// (the generator's Weyl sequence), tabulated once on the host.
struct PhiloxKeys {
  uint32_t k[10][2];
};

struct EvalParams {
  int mode;                   // CCS_EXACT / CCS_SAMPLED / CCS_STITCH
  uint32_t shots, seed_lo, seed_hi;
  PhiloxKeys keys;            // round keys of (seed_lo, seed_hi)
  int keep_tableaus;
  int shared_body;            // 1: variants start from their fragment's body tableau
  int screen;                 // 1: the screen finishes every Clifford variant (no tableau kernel)
  int hub_sampler;            // host only: the caller's hub sampler choice (0 automatic)
  double inv_shots;
};

// Read view of a hub's contraction operand (Q^T, row-major K x M) from
// float index `off` of TQ on: FP32, or int16 count sums times the scale.
struct HubView {
  const float* f;
  const int16_t* h;
  float scale;
  __device__ __forceinline__ float at(long long i) const { return h ? (float)h[i] * scale : f[i]; }
};
__device__ __forceinline__ HubView hub_view(const DevRes& R, const FragDev& H, long long off) {
  HubView v;
  v.f = R.TQ + off;
  v.h = (R.hub_i16 && H.clifford) ? reinterpret_cast<const int16_t*>(R.TQ + H.T_off) + (off - H.T_off) : nullptr;
  v.scale = R.hub_scale;
  return v;
}

// Kernels the library has launched in this process; a replayed CUDA graph
// adds its kernel nodes once per replay.
void note_launch();
void note_launches(long long n);
long long launch_count();

// Kernel launchers (stream-ordered; return cudaError_t of the launch).
// words_per_op: 64-row words of one fused op a thread updates (1, 2, 4 or 8)
// Body tableau of every Clifford fragment (identity evolved by the gate
// sequence, no preparations or basis changes), one CTA per 64-row word.
// With basis set, a second launch writes the shared-row bases and the Z
// images the screen needs.
cudaError_t launch_body(const DevPlan& p, const DevRes& r, int smem_optin, bool basis, cudaStream_t s);
// Screen of every Clifford variant from its fragment's shared-row basis and
// Z images: outcome space (rank, reduced basis, offset) and Z-string values,
// without a tableau per variant.  Used unless tableaus are kept; then the
// tableau kernel (launch_clifford) takes every variant instead.
cudaError_t launch_screen(const DevPlan& p, const DevRes& r, const EvalParams& e, int sm_count, int smem_optin,
                          cudaStream_t s);
cudaError_t launch_clifford(const DevPlan& p, const DevRes& r, const EvalParams& e,
                            int threads, int words_per_op, int smem_words, int grid, cudaStream_t s);
cudaError_t launch_sample(const DevPlan& p, const DevRes& r, const EvalParams& e, const int2* items,
                          int n_items, int shots_per_cta, int threads, cudaStream_t s);
// Sampling + output fold of star hubs (one CTA per hub variant); writes the
// hub's contraction operand Q into TQ, and dense counts if keep_counts.
// bytes_ok: every hub has >= 2 marginal bits, <= 4 quantum outputs and |A| <= 16
// (the byte-counter kernel applies)
cudaError_t launch_sample_hub(const DevPlan& p, const DevRes& r, const EvalParams& e, const int2* items,
                              int n_items, int max_nA, int threads, int keep_counts, bool bytes_ok, cudaStream_t s);
// Stitched mode: the contraction operand of Clifford hubs in closed form from
// each variant's outcome space (one CTA per hub variant), with the row flags.
cudaError_t launch_hub_exact(const DevPlan& p, const DevRes& r, const int2* items, int n_items, cudaStream_t s);
cudaError_t launch_statevector(const DevPlan& p, const DevRes& r, int max_n, int threads,
                               int grid, cudaStream_t s);
// A subset of fragments to fold: fidx[i] is the FragDev index of segment i;
// t_prefix (nf + 1 entries) counts T_f entries.
struct FoldSet {
  const int* fidx;
  const long long* t_prefix;
  int nf;
  long long total;
};
cudaError_t launch_fold(const DevPlan& p, const DevRes& r, const EvalParams& e, const FoldSet& f,
                        cudaStream_t s);
// Maximum-likelihood correction of fragment models (Sec. V-C).  One record
// per fragment to correct; fragments with the same number of cut slots d
// form a group (one launch of the per-block kernels).
struct MlFrag {
  int frag;                // FragDev index
  int d;                   // cut slots (the Choi block has D = 2^d rows)
  int hub;                 // 1: a star hub (its operand Q^T is read and rewritten as well)
  int i16;                 // the hub operand holds int16 count sums (value = sum x hub_scale)
  int index;               // position in the launch's record list (its threshold)
  long long blk0;          // first block (outcome 0) of the fragment within its group
  long long ev_off;        // float index of its 2^m x D eigenvalues in the scratch
  long long vec_off;       // float index of its 2^m x D x D complex64 eigenvector entries
  double total;            // the eigenvalues' sum after the correction: 2^qin
};
struct MlGroup {
  int d, first, count;     // cut slots; range of MlFrag records
  long long blocks;        // sum of 2^m over them
};
// Eigendecomposition of every block, the threshold per fragment, and the
// rebuilt T_f (and hub operands); d <= 6.  `scratch` holds the eigenvalues
// and eigenvectors, `theta` one double per record.
cudaError_t launch_ml_correct(const DevPlan& p, const DevRes& r, const MlFrag* d_frags, int n_frags,
                              const MlGroup* groups, int n_groups, float* scratch, double* theta, cudaStream_t s);
constexpr int kMlMaxSlots = 6;

// Contraction operands of star problems: Q of each hub from its variant data
// (set `hubs`) and T' of every other fragment from its T (set `others`).
cudaError_t launch_operands(const DevPlan& p, const DevRes& r, const EvalParams& e, const FoldSet& hubs,
                            const FoldSet& others, cudaStream_t s);
// Recombination of every star problem: R build, split-K GEMM, FP64 reduce
// and scatter into marg_out (2^n_marg doubles per problem at marg_off), and
// the Z-string contraction into zexp_out.  `scratch` holds R and the split-K
// partials (r_total + part_total floats).
// A range [lo, hi) of the cut index P summed by a partial contraction
// (hi < 0: to the end); every problem clamps it to its own 4^k.
struct KRange {
  long long lo, hi;
  __host__ __device__ long long lo_of(long long K) const { return lo < K ? lo : K; }
  __host__ __device__ long long hi_of(long long K) const { return hi < 0 || hi > K ? K : hi; }
  __host__ __device__ bool full() const { return lo == 0 && hi < 0; }
};

struct RecombSizes {
  long long r_total, part_total, gemm_blocks, out_total, z_total;
  const int2* direct_items;      // (problem, hub-output slice) contracted leaf by leaf, one CTA each
  int n_direct;
  int direct_stage_floats;       // floats of each of the two intermediate buffers
  int chain;                     // 1: some problem takes the R / GEMM / reduce chain
  const long long* r_prefix;     // per problem, K*N entries
  const long long* blk_prefix;   // per problem, GEMM blocks
  const long long* out_prefix;   // per problem, M*N outputs
  const long long* z_prefix;     // per problem, Z-strings
  int max_tile_smem;             // bytes of dynamic shared memory per GEMM block
  const ProblemDev* host_problems;   // host copy of the problems (per-problem GEMM launches)
  int n_problems;
  uint16_t* rt_scratch;          // bf16 R'^T of problems eligible for the tensor-core GEMM
  int tensor_cores;              // 1: BF16 contractions of eligible problems on tcgen05
  int stitched;                  // 1: Clifford hubs' operand rows flagged in DevRes::qnz (zero rows
                                 //    of streamed problems are neither written nor read)
  KRange krange;                 // the cut-index terms summed ({0, -1}: all)
  int has_general;               // 1: some problem is not a star
};
cudaError_t launch_recombine(const DevPlan& p, const DevRes& r, int precision, const RecombSizes& z,
                             float* scratch, double* marg_out, double* zexp_out, cudaStream_t s);
// context stream; learned scorer helpers (mpnn.cu, features.cpp)
cudaStream_t c_stream(ccs_ctx c);
int mpnn_predict(ccs_mpnn n, const ccs_graph_batch* b, float* pred);
int featurize(const Problem& p, const std::vector<ccs_cut>& cuts, std::vector<float>& x, std::vector<int>& rowptr,
              std::vector<int>& col, std::vector<float>& val, std::vector<float>& val_t, std::vector<float>& glob,
              std::string& err);
// tcgen05 GEMM (gemm_tc.cu): partials[split][m][n] of A (M x K) x Bt^T (Bt: N x K), bf16
bool gemm_tc_supported(int M, int N, long long K);
cudaError_t launch_gemm_tc(const void* A, const void* Bt, int M, int N, long long K, int splits, float* partials,
                           unsigned* status, cudaStream_t s);

}  // namespace ccs
