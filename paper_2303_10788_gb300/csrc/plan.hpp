// Host-side plan of the circuit-cutting hot path: fragments, variants and the
// compiled gate streams the device kernels consume.
#pragma once

#include <algorithm>
#include <array>
#include <complex>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "ccs.h"

namespace ccs {

// Limits of the device kernels.
constexpr int kMaxMeas = 24;        // |A_f|: dense 2^|A_f| outcome tables
constexpr int kMaxNCWidth = 12;     // complex64 statevector of 2^12 amplitudes in smem
constexpr int kMaxTableauQubits = 640;  // per-variant tableaus: (2n+3) x 2*ceil(n/64) words fit 227 KB of smem
// Clifford fragments on the shared-body path (the default: one body per
// fragment, kept in global memory, one 64-row word per column in a CTA's
// shared memory; no per-variant tableau): a warp covers its 2*ceil(n/64) words.
constexpr int kMaxBodyQubits = 1024;
constexpr int kMaxCuts = 12;
constexpr int kMaxProblemFragments = kMaxCuts + 1;   // fragments of one problem (the contraction stages them)
constexpr int kMaxMarginal = 24;
// Circuit size accepted at the ABI (host arrays are linear in both).
constexpr uint32_t kMaxCircuitQubits = 1u << 24;
constexpr uint32_t kMaxCircuitGates = 1u << 30;

// Internal opcode of a Z^a gate with 2a = 0 mod 4 (the identity): kept as a
// gate so that cut positions, which are gate indices, stay valid.
constexpr int kOpI = 64;

inline bool is_nonclifford_op(int op) { return op == CCS_T || op == CCS_TDG || op == CCS_ZPOW; }

// The ABI gate list as (op, q0, q1) triples (q1 = -1 for one-qubit gates) and
// per-gate exponents: Z^a with 2a an integer becomes the Clifford S^{2a}
// (kOpI, S, Z or SDG, Sec. II-C); any other Z^a stays CCS_ZPOW with its
// exponent reduced mod 2 in `gparam` (0 for every other gate).
int load_gates(const ccs_gate* g, uint32_t n_gates, std::vector<std::array<int, 3>>& gates,
               std::vector<double>& gparam, std::string& err);

// CCS_OK, or INVALID_ARG for an empty circuit, a null gate list or a size
// beyond kMaxCircuitQubits / kMaxCircuitGates.
int check_circuit(const ccs_problem& q, std::string& err);

// A fused one- or two-qubit Clifford conjugation acting on the bit-sliced
// columns (x_a, z_a, x_b, z_b) = (v0, v1, v2, v3):
//   u_i = XOR_j M[i][j] v_j            (M bit 4*i + j)
//   r  ^= XOR_S anf[S] prod_{j in S} v_j   (algebraic normal form of the sign flip)
// One-qubit ops use the all-zero dummy column pair as b.
struct CliffordOp {
  uint16_t qa, qb, M, anf;
};
static_assert(sizeof(CliffordOp) == 8, "packed op");

// A fused non-Clifford-fragment op: 2x2 (one qubit) or 4x4 (two qubits,
// basis index = bit_a + 2 bit_b) complex unitary, stored row-major.
struct NCOp {
  int32_t a, b;          // b < 0 for one-qubit ops
  float m[32];           // re, im interleaved
};

struct Frag {
  int problem = 0, index = 0;
  bool clifford = true;
  std::vector<std::pair<uint32_t, uint32_t>> wires;  // (qubit, segment)
  std::vector<std::array<int, 3>> gates;             // (op, a, b), local wires
  std::vector<double> gparam;                        // per gate: Z^a exponent, else 0 (empty: all 0)
  std::vector<int> qin_cut, qin_wire, qout_cut, qout_wire;
  std::vector<int> marg_pos, marg_wire;
  std::vector<int> slots;       // incident cut ids, ascending
  std::vector<int> slot_kind;   // 0 = quantum input, 1 = quantum output
  std::vector<int> slot_idx;    // index into qin_* / qout_*
  std::vector<std::vector<int>> zwires;   // per Z-string: wires carrying its qubits' outputs
  // compiled streams
  std::vector<CliffordOp> cops;
  std::vector<int> moment_start;          // n_moments + 1 entries into cops / nops
  std::vector<NCOp> nops;

  int n() const { return (int)wires.size(); }
  int n_variants() const {
    int v = 1;
    for (size_t i = 0; i < qin_wire.size(); ++i) v *= 4;
    for (size_t i = 0; i < qout_wire.size(); ++i) v *= 3;
    return v;
  }
  int n_meas() const { return (int)(marg_wire.size() + qout_wire.size()); }
  int n_moments() const { return moment_start.empty() ? 0 : (int)moment_start.size() - 1; }
};

struct Problem {
  uint32_t n_qubits = 0;
  std::vector<std::array<int, 3>> gates;
  std::vector<double> gparam;    // per gate: Z^a exponent, else 0 (may be empty: all 0)
  std::vector<ccs_cut> cuts;     // canonical order
  std::vector<uint32_t> marginal;
  std::vector<std::vector<uint32_t>> zstrings;
  std::vector<int> frag_ids;     // into Plan::frags
  int hub = -1;                  // local fragment index of the star's hub, -1 if not a star
};

// Union-find over wire segments; the root of a set is its smallest member.
struct UF {
  std::vector<int> p;
  explicit UF(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int find(int x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
  }
  void join(int a, int b) {
    a = find(a); b = find(b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  }
};

// Fragment a problem at its cuts (the cuts must already be canonical).
// Returns CCS_OK or an error code with `err` set.
int fragment_problem(Problem& p, int problem_index, std::vector<Frag>& out, std::string& err);

// Fuse the fragment's gates into moments of CliffordOp / NCOp.
void compile_clifford(Frag& f);
void compile_nc(Frag& f);

// One-qubit fused ops for the variant prologue / epilogue (on qubit 0,
// dummy b): preparations |0>,|1>,|+>,|+i> and bases X, Y, Z.
CliffordOp prep_op(int s);
CliffordOp basis_op(int b);
void prep_matrix(int s, float out[8]);
void basis_matrix(int b, float out[8]);

// Greedy cut search (Sec. V-A: cuts isolate the non-Clifford operations).
struct CutSearchOpts {
  int max_cuts = kMaxCuts;
  int max_nc_width = 10;
};
struct CutCandidate {
  std::vector<ccs_cut> cuts;
  double cost = 0.0;
  std::vector<int> region_of_qubit;   // diagnostic
};
int greedy_cuts(const Problem& p, const CutSearchOpts& o, std::vector<CutCandidate>& cands,
                std::string& err);
double plan_cost(const Problem& p, const std::vector<ccs_cut>& cuts, bool* ok);

// The learned scorer's input graph: the candidate-independent interaction
// graph (CSR of A = D^-1 Adj and of A^T's values, per-qubit gate counts)
// once per circuit, the node and global features per candidate cut set.
struct GraphBase {
  std::vector<int> rowptr, col, tcount, gcount;
  std::vector<float> val, val_t;
};
GraphBase graph_base(const Problem& p);
int featurize_nodes(const Problem& p, const GraphBase& g, const std::vector<ccs_cut>& cuts, std::vector<float>& x,
                    std::vector<float>& glob, std::string& err);

}  // namespace ccs
