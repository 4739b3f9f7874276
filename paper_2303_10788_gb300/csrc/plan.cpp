// Fragmenting (Sec. V-A), variant bookkeeping (Sec. V-B) and gate-stream
// compilation for the device kernels.
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace ccs {

namespace {

bool is_two_qubit(int op) { return op == CCS_CX || op == CCS_CZ; }
bool is_clifford_op(int op) { return (op >= CCS_H && op <= CCS_CZ) || op == kOpI; }

// CHP update (Sec. III of Aaronson-Gottesman) of the local Pauli patterns
// (x_a, z_a, x_b, z_b) and their signs, 16 patterns at once: bit v of each
// plane is the x_a, z_a, x_b, z_b or sign bit of pattern v.
void chp_planes(int op, int ra, int rb, uint32_t x[2], uint32_t z[2], uint32_t& flip) {
  const uint32_t ONE = 0xffffu;
  switch (op) {
    case CCS_H: flip ^= x[ra] & z[ra]; std::swap(x[ra], z[ra]); break;
    case CCS_S: flip ^= x[ra] & z[ra]; z[ra] ^= x[ra]; break;
    case CCS_SDG: flip ^= x[ra] & (z[ra] ^ ONE); z[ra] ^= x[ra]; break;
    case CCS_X: flip ^= z[ra]; break;
    case CCS_Y: flip ^= x[ra] ^ z[ra]; break;
    case CCS_Z: flip ^= x[ra]; break;
    case CCS_CX:
      flip ^= x[ra] & z[rb] & (x[rb] ^ z[ra] ^ ONE);
      x[rb] ^= x[ra];
      z[ra] ^= z[rb];
      break;
    case CCS_CZ:
      flip ^= x[ra] & x[rb] & (z[ra] ^ z[rb]);
      z[ra] ^= x[rb];
      z[rb] ^= x[ra];
      break;
    default: break;
  }
}

// The one-qubit Cliffords of the gate set as plane updates without a branch:
// x' = (x & P) ^ (z & Q), z' = (x & R) ^ (z & S),
// flip ^= (x & z & A) ^ (x & B) ^ (z & C)   (all-ones or zero masks;
// the same rules as chp_planes: H swaps x and z, S and S^dagger add x to z,
// the Paulis only flip signs).  Row = opcode H..Z, then the identity.
struct OneQubitRule { uint32_t P, Q, R, S, A, B, C; };
constexpr uint32_t kOnes = 0xffffu;
constexpr OneQubitRule kOneQubit[7] = {
    {0, kOnes, kOnes, 0, kOnes, 0, 0},          // H
    {kOnes, 0, kOnes, kOnes, kOnes, 0, 0},      // S
    {kOnes, 0, kOnes, kOnes, kOnes, kOnes, 0},  // S^dagger: flip ^= x & ~z
    {kOnes, 0, 0, kOnes, 0, 0, kOnes},          // X
    {kOnes, 0, 0, kOnes, 0, kOnes, kOnes},      // Y
    {kOnes, 0, 0, kOnes, 0, kOnes, 0},          // Z
    {kOnes, 0, 0, kOnes, 0, 0, 0},              // identity
};
inline void one_qubit_planes(int op, uint32_t& x, uint32_t& z, uint32_t& flip) {
  const OneQubitRule& r = kOneQubit[op == kOpI ? 6 : op];
  flip ^= (x & z & r.A) ^ (x & r.B) ^ (z & r.C);
  const uint32_t nx = (x & r.P) ^ (z & r.Q), nz = (x & r.R) ^ (z & r.S);
  x = nx;
  z = nz;
}

// Identity planes: pattern v has x_a = bit 0, z_a = bit 1, x_b = bit 2, z_b = bit 3 of v.
constexpr uint32_t kPX0 = 0xaaaau, kPX1 = 0xf0f0u, kPZ0 = 0xccccu, kPZ1 = 0xff00u;

// (M, anf) of the Clifford update given by its 16-pattern planes: column j
// of M is the image of the unit pattern 1 << j (bit i of plane i at that
// pattern), and the sign polynomial's algebraic normal form is the Moebius
// transform of the 16-entry flip truth table (a[s] = XOR of f[t], t a subset
// of s), done on the 16-bit word one variable at a time.
CliffordOp clifford_from_planes(const uint32_t x[2], const uint32_t z[2], uint32_t flip) {
  CliffordOp op{0, 0, 0, 0};
  const uint32_t planes[4] = {x[0], z[0], x[1], z[1]};
  uint32_t M = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) M |= ((planes[i] >> (1u << j)) & 1u) << (4 * i + j);
  op.M = (uint16_t)M;
  uint32_t a = flip & 0xffffu;
  a ^= (a << 1) & 0xaaaau;
  a ^= (a << 2) & 0xccccu;
  a ^= (a << 4) & 0xf0f0u;
  a ^= (a << 8) & 0xff00u;
  op.anf = (uint16_t)a;
  return op;
}

// (M, anf) of a gate word acting on roles 0 (= a) and 1 (= b).
CliffordOp clifford_from_word(const std::vector<std::array<int, 3>>& word) {
  uint32_t x[2] = {kPX0, kPX1}, z[2] = {kPZ0, kPZ1}, flip = 0;
  for (auto& g : word) chp_planes(g[0], g[1], g[2] < 0 ? 1 - g[1] : g[2], x, z, flip);
  return clifford_from_planes(x, z, flip);
}

using cd = std::complex<double>;

void gate_matrix_1q(int op, double param, cd m[4]) {
  const double r = 1.0 / std::sqrt(2.0);
  const cd I(0, 1);
  cd id[4] = {1, 0, 0, 1};
  for (int i = 0; i < 4; ++i) m[i] = id[i];
  switch (op) {
    case CCS_H: m[0] = r; m[1] = r; m[2] = r; m[3] = -r; break;
    case CCS_S: m[3] = I; break;
    case CCS_SDG: m[3] = -I; break;
    case CCS_X: m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0; break;
    case CCS_Y: m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0; break;
    case CCS_Z: m[3] = -1; break;
    case CCS_T: m[3] = std::polar(1.0, M_PI / 4); break;
    case CCS_TDG: m[3] = std::polar(1.0, -M_PI / 4); break;
    case CCS_ZPOW: m[3] = std::polar(1.0, M_PI * param); break;   // Z^a = diag(1, e^{i pi a})
    default: break;                                                // kOpI: identity
  }
}

// One gate of a fused op's word: opcode, roles (rb < 0: one-qubit), exponent.
struct WordGate {
  int op, ra, rb;
  double param;
};

// rows (u0, u1) <- G (u0, u1) for a one-qubit gate G, n entries per row: the
// Paulis, S, S^dagger and the identity as exact permutations / sign and
// i-multiples, the phase gates on u1 only, H as r(u0 + u1), r(u0 - u1);
// other gates as the full 2x2 product.
void mix_rows(int op, double param, cd* u0, cd* u1, int n) {
  switch (op) {
    case kOpI: return;
    case CCS_X:
      for (int j = 0; j < n; ++j) std::swap(u0[j], u1[j]);
      return;
    case CCS_Y:
      for (int j = 0; j < n; ++j) {
        const cd a = u0[j], b = u1[j];
        u0[j] = cd(b.imag(), -b.real());     // -i b
        u1[j] = cd(-a.imag(), a.real());     //  i a
      }
      return;
    case CCS_Z:
      for (int j = 0; j < n; ++j) u1[j] = -u1[j];
      return;
    case CCS_S:
      for (int j = 0; j < n; ++j) u1[j] = cd(-u1[j].imag(), u1[j].real());
      return;
    case CCS_SDG:
      for (int j = 0; j < n; ++j) u1[j] = cd(u1[j].imag(), -u1[j].real());
      return;
    case CCS_T: case CCS_TDG: case CCS_ZPOW: {
      cd G[4];
      gate_matrix_1q(op, param, G);
      for (int j = 0; j < n; ++j) u1[j] = G[3] * u1[j];
      return;
    }
    case CCS_H: {
      const double r = 1.0 / std::sqrt(2.0);
      for (int j = 0; j < n; ++j) {
        const cd a = u0[j], b = u1[j];
        u0[j] = r * a + r * b;
        u1[j] = r * a - r * b;
      }
      return;
    }
    default: {
      cd G[4];
      gate_matrix_1q(op, param, G);
      for (int j = 0; j < n; ++j) {
        const cd a = u0[j], b = u1[j];
        u0[j] = G[0] * a + G[1] * b;
        u1[j] = G[2] * a + G[3] * b;
      }
    }
  }
}

// A fused op of a Clifford fragment: each gate is applied to the op's
// 16-pattern planes as it arrives, so no gate word is stored.
struct PlaneOp {
  int a, b;                                   // b < 0: one-qubit op
  uint32_t px[2], pz[2], pf;
  bool dead;
  PlaneOp(int qa, int qb) : a(qa), b(qb), px{kPX0, kPX1}, pz{kPZ0, kPZ1}, pf(0), dead(false) {}
  void add(int op, int ra, int rb, double) {
    if (rb < 0 && op <= CCS_Z) one_qubit_planes(op, px[ra], pz[ra], pf);
    else if (rb < 0 && op == kOpI) return;
    else chp_planes(op, ra, rb < 0 ? 1 - ra : rb, px, pz, pf);
  }
};
// A fused op of a statevector fragment keeps its gate word (for the unitary).
struct WordOp {
  int a, b;
  std::vector<WordGate> word;
  bool dead = false;
  WordOp(int qa, int qb) : a(qa), b(qb) {}
  void add(int op, int ra, int rb, double param) { word.push_back({op, ra, rb, param}); }
};

// The op made of a trailing one-qubit op on each side (either may be
// absent) followed by the two-qubit gate's roles.
inline void absorb(PlaneOp& nf, const PlaneOp* g0, const PlaneOp* g1) {
  if (!g0 && !g1) return;
  // A one-qubit op's planes hold its images of the patterns w = 0..3 in
  // bits 0..3.  Role 0 reads w from bits 0-1 of the two-qubit pattern v
  // (the 4-bit image repeated in every nibble), role 1 from bits 2-3
  // (bit k of the image filling nibble k).
  auto rep = [](uint32_t t) { t &= 0xfu; return t * 0x1111u; };
  auto spread = [](uint32_t t) {
    return ((t & 1u) ? 0x000fu : 0u) | ((t & 2u) ? 0x00f0u : 0u) | ((t & 4u) ? 0x0f00u : 0u) |
           ((t & 8u) ? 0xf000u : 0u);
  };
  nf.px[0] = g0 ? rep(g0->px[0]) : kPX0;
  nf.pz[0] = g0 ? rep(g0->pz[0]) : kPZ0;
  nf.px[1] = g1 ? spread(g1->px[0]) : kPX1;
  nf.pz[1] = g1 ? spread(g1->pz[0]) : kPZ1;
  nf.pf = (g0 ? rep(g0->pf) : 0u) ^ (g1 ? spread(g1->pf) : 0u);
}
inline void absorb(WordOp& nf, WordOp* g0, WordOp* g1) {
  for (int side = 0; side < 2; ++side) {
    WordOp* g = side == 0 ? g0 : g1;
    if (!g) continue;
    for (auto& w : g->word) nf.word.push_back({w.op, side, -1, w.param});
    g->word.clear();
  }
}

// Fuse consecutive gates per qubit (pair) and assign ASAP moments: on return
// order[start[L] .. start[L+1]) are the live ops of moment L (indices into
// ops, in creation order).
template <class Op>
void fuse_and_layer(const Frag& f, std::vector<Op>& ops, std::vector<int>& order, std::vector<int>& start) {
  const int n = f.n();
  std::vector<int> last(n, -1);
  for (size_t gi = 0; gi < f.gates.size(); ++gi) {
    const auto& g = f.gates[gi];
    const int op = g[0], a = g[1], b = g[2];
    const double prm = f.gparam.empty() ? 0.0 : f.gparam[gi];
    if (!is_two_qubit(op)) {
      if (last[a] >= 0) {
        Op& F = ops[last[a]];
        F.add(op, F.a == a ? 0 : 1, -1, prm);
      } else {
        ops.emplace_back(a, -1);
        ops.back().add(op, 0, -1, prm);
        last[a] = (int)ops.size() - 1;
      }
      continue;
    }
    const int la = last[a], lb = last[b];
    if (la >= 0 && la == lb) {
      Op& F = ops[la];
      const int ra = F.a == a ? 0 : 1;
      F.add(op, ra, 1 - ra, 0.0);
      continue;
    }
    Op* g1[2] = {nullptr, nullptr};
    for (int side = 0; side < 2; ++side) {
      const int lq = side == 0 ? la : lb;
      if (lq >= 0 && ops[lq].b < 0) {     // absorb a trailing one-qubit op
        g1[side] = &ops[lq];
        ops[lq].dead = true;
      }
    }
    ops.emplace_back(a, b);                  // capacity reserved: g1 stays valid
    Op& nf = ops.back();
    absorb(nf, g1[0], g1[1]);
    nf.add(op, 0, 1, 0.0);
    last[a] = last[b] = (int)ops.size() - 1;
  }
  std::vector<int> layer_of_q(n, -1), lay(ops.size(), -1);
  int nl = 0;
  for (size_t i = 0; i < ops.size(); ++i) {
    const Op& F = ops[i];
    if (F.dead) continue;
    int L = layer_of_q[F.a];
    if (F.b >= 0) L = std::max(L, layer_of_q[F.b]);
    L += 1;
    layer_of_q[F.a] = L;
    if (F.b >= 0) layer_of_q[F.b] = L;
    lay[i] = L;
    nl = std::max(nl, L + 1);
  }
  start.assign(nl + 1, 0);                     // counting sort by moment, stable
  for (int L : lay)
    if (L >= 0) ++start[L + 1];
  for (int L = 0; L < nl; ++L) start[L + 1] += start[L];
  order.resize(start[nl]);
  std::vector<int> fill(start.begin(), start.end() - 1);
  for (size_t i = 0; i < ops.size(); ++i)
    if (lay[i] >= 0) order[fill[lay[i]]++] = (int)i;
}

}  // namespace

int check_circuit(const ccs_problem& q, std::string& err) {
  if (q.n_qubits == 0 || (q.n_gates && !q.gates)) { err = "empty circuit"; return CCS_ERR_INVALID_ARG; }
  if (q.n_qubits > kMaxCircuitQubits) { err = "too many qubits"; return CCS_ERR_INVALID_ARG; }
  if (q.n_gates > kMaxCircuitGates) { err = "too many gates"; return CCS_ERR_INVALID_ARG; }
  return CCS_OK;
}

int load_gates(const ccs_gate* G, uint32_t ng, std::vector<std::array<int, 3>>& gates,
               std::vector<double>& gparam, std::string& err) {
  static const int kSPow[4] = {kOpI, CCS_S, CCS_Z, CCS_SDG};   // S^0 .. S^3
  gates.resize(ng);
  gparam.clear();                    // sized only when a non-Clifford exponent appears (empty: all 0)
  for (uint32_t i = 0; i < ng; ++i) {
    const ccs_gate& g = G[i];
    if (g.op > CCS_ZPOW) { err = "unknown gate opcode"; return CCS_ERR_UNSUPPORTED_GATE; }
    int op = g.op;
    if (op == CCS_ZPOW) {
      const double k = 2.0 * g.param;
      if (!std::isfinite(k)) { err = "Z^a exponent not finite"; return CCS_ERR_INVALID_ARG; }
      if (k == std::floor(k)) {
        double m = std::fmod(k, 4.0);       // exact for every integral double
        if (m < 0) m += 4.0;
        op = kSPow[(int)m];
      } else {
        double a = std::fmod(g.param, 2.0);  // e^{i pi a} has period 2 in a
        if (a < 0) a += 2.0;
        if (gparam.empty()) gparam.assign(ng, 0.0);
        gparam[i] = a;
      }
    }
    const bool two = op == CCS_CX || op == CCS_CZ;
    gates[i] = {op, (int)g.q[0], two ? (int)g.q[1] : -1};
  }
  return CCS_OK;
}

int fragment_problem(Problem& p, int pi, std::vector<Frag>& out, std::string& err) {
  const int n = (int)p.n_qubits;
  const int ng = (int)p.gates.size();
  if (!p.gparam.empty() && (int)p.gparam.size() != ng) { err = "gate exponent list size"; return CCS_ERR_INVALID_ARG; }
  for (auto& c : p.cuts)
    if ((int)c.qubit >= n || (int)c.gate_index > ng) { err = "cut out of range"; return CCS_ERR_INVALID_ARG; }
  std::sort(p.cuts.begin(), p.cuts.end(), [](const ccs_cut& x, const ccs_cut& y) {
    return x.gate_index != y.gate_index ? x.gate_index < y.gate_index : x.qubit < y.qubit;
  });
  for (size_t i = 1; i < p.cuts.size(); ++i)
    if (p.cuts[i].qubit == p.cuts[i - 1].qubit && p.cuts[i].gate_index == p.cuts[i - 1].gate_index) {
      err = "duplicate cut"; return CCS_ERR_INVALID_ARG;
    }
  if ((int)p.cuts.size() > kMaxCuts) { err = "too many cuts"; return CCS_ERR_TOO_MANY_CUTS; }
  if (p.marginal.size() > (size_t)kMaxMarginal) { err = "marginal too wide"; return CCS_ERR_INVALID_ARG; }
  for (auto q : p.marginal)
    if ((int)q >= n) { err = "marginal qubit out of range"; return CCS_ERR_INVALID_ARG; }
  for (size_t i = 0; i < p.marginal.size(); ++i)
    for (size_t j = 0; j < i; ++j)
      if (p.marginal[i] == p.marginal[j]) { err = "repeated marginal qubit"; return CCS_ERR_INVALID_ARG; }

  std::vector<std::vector<int>> pos(n);
  for (auto& c : p.cuts) pos[c.qubit].push_back((int)c.gate_index);
  std::vector<int> base(n + 1, 0);
  for (int q = 0; q < n; ++q) base[q + 1] = base[q] + (int)pos[q].size() + 1;
  // Each qubit's current segment while walking the gates: a cut (q, g) starts
  // q's next segment at gate g.  The cuts are sorted by gate index, so one
  // cursor over them moves every qubit's segment forward; each pass over the
  // gates replays it (no per-gate segment arrays).
  thread_local std::vector<int> segcur;
  auto walk = [&](auto&& visit) {
    segcur.assign(base.begin(), base.end() - 1);
    size_t nc = 0;
    for (int gi = 0; gi < ng; ++gi) {
      while (nc < p.cuts.size() && (int)p.cuts[nc].gate_index <= gi) ++segcur[p.cuts[nc++].qubit];
      const auto& g = p.gates[gi];
      visit(gi, g, segcur[g[1]], is_two_qubit(g[0]) ? segcur[g[2]] : -1);
    }
  };
  // first pass: check each gate, join the segments a two-qubit gate touches
  // and count the gates per segment (a gate belongs to its first operand's)
  UF uf(base[n]);
  std::vector<int> seg_gates(base[n], 0);
  {
    segcur.assign(base.begin(), base.end() - 1);
    size_t nc = 0;
    for (int gi = 0; gi < ng; ++gi) {
      while (nc < p.cuts.size() && (int)p.cuts[nc].gate_index <= gi) ++segcur[p.cuts[nc++].qubit];
      const auto& g = p.gates[gi];
      if (g[0] < 0 || (g[0] > CCS_ZPOW && g[0] != kOpI)) { err = "unknown gate opcode"; return CCS_ERR_UNSUPPORTED_GATE; }
      if (g[1] < 0 || g[1] >= n) { err = "gate qubit out of range"; return CCS_ERR_INVALID_ARG; }
      const int sa = segcur[g[1]];
      ++seg_gates[sa];
      if (is_two_qubit(g[0])) {
        if (g[2] < 0 || g[2] >= n || g[2] == g[1]) { err = "bad two-qubit gate operands"; return CCS_ERR_INVALID_ARG; }
        uf.join(sa, segcur[g[2]]);
      }
    }
  }
  // fragments ordered by first wire; wires by (qubit, segment) = segment id
  std::vector<int> root_to_frag(base[n], -1);
  std::vector<std::pair<int, int>> where(base[n]);
  const int first = (int)out.size();
  for (int q = 0, s = 0; q < n; ++q)
    for (; s < base[q + 1]; ++s) {
      const int r = uf.find(s);
      if (root_to_frag[r] < 0) {
        root_to_frag[r] = (int)out.size();
        Frag f;
        f.problem = pi;
        f.index = (int)out.size() - first;
        out.push_back(std::move(f));
      }
      Frag& f = out[root_to_frag[r]];
      where[s] = {root_to_frag[r], f.n()};
      f.wires.push_back({(uint32_t)q, (uint32_t)(s - base[q])});
    }
  // second pass: every gate written to its fragment's pre-sized list
  const int nfr = (int)out.size() - first;
  std::vector<std::array<int, 3>*> gdst(nfr);
  std::vector<double*> pdst(nfr, nullptr);
  {
    std::vector<int> count(nfr, 0);
    for (int s = 0; s < base[n]; ++s) count[where[s].first - first] += seg_gates[s];
    for (int fi = 0; fi < nfr; ++fi) {
      out[first + fi].gates.resize(count[fi]);
      gdst[fi] = out[first + fi].gates.data();
      if (!p.gparam.empty()) {
        out[first + fi].gparam.resize(count[fi]);
        pdst[fi] = out[first + fi].gparam.data();
      }
    }
  }
  walk([&](int gi, const std::array<int, 3>& g, int sa, int sb) {
    const auto wa = where[sa];
    const int fl = wa.first - first;
    *gdst[fl]++ = {g[0], wa.second, sb >= 0 ? where[sb].second : -1};
    if (pdst[fl]) *pdst[fl]++ = sb >= 0 ? 0.0 : p.gparam[gi];
    if (sb < 0 && !is_clifford_op(g[0])) out[wa.first].clifford = false;
  });
  for (int ci = 0; ci < (int)p.cuts.size(); ++ci) {
    int q = p.cuts[ci].qubit;
    int k = (int)(std::find(pos[q].begin(), pos[q].end(), (int)p.cuts[ci].gate_index) - pos[q].begin()) + 1;
    auto up = where[base[q] + k - 1], dn = where[base[q] + k];
    if (up.first == dn.first) {
      err = "a cut whose two ends lie in one fragment is not supported";
      return CCS_ERR_UNSUPPORTED;
    }
    out[up.first].qout_cut.push_back(ci);
    out[up.first].qout_wire.push_back(up.second);
    out[dn.first].qin_cut.push_back(ci);
    out[dn.first].qin_wire.push_back(dn.second);
  }
  for (int mi = 0; mi < (int)p.marginal.size(); ++mi) {
    int q = p.marginal[mi];
    auto w = where[base[q] + (int)pos[q].size()];
    out[w.first].marg_pos.push_back(mi);
    out[w.first].marg_wire.push_back(w.second);
  }
  for (int fi = first; fi < (int)out.size(); ++fi) {
    Frag& f = out[fi];
    f.zwires.assign(p.zstrings.size(), {});
    std::vector<std::pair<int, std::pair<int, int>>> sl;
    for (size_t j = 0; j < f.qin_cut.size(); ++j) sl.push_back({f.qin_cut[j], {0, (int)j}});
    for (size_t j = 0; j < f.qout_cut.size(); ++j) sl.push_back({f.qout_cut[j], {1, (int)j}});
    std::sort(sl.begin(), sl.end());
    for (auto& e : sl) {
      f.slots.push_back(e.first);
      f.slot_kind.push_back(e.second.first);
      f.slot_idx.push_back(e.second.second);
    }
  }
  for (size_t si = 0; si < p.zstrings.size(); ++si)
    for (auto q : p.zstrings[si]) {
      if ((int)q >= n) { err = "Z-string qubit out of range"; return CCS_ERR_INVALID_ARG; }
      auto w = where[base[q] + (int)pos[q].size()];
      out[w.first].zwires[si].push_back(w.second);
    }
  p.frag_ids.clear();
  for (int fi = first; fi < (int)out.size(); ++fi) {
    Frag& f = out[fi];
    if (!f.clifford && f.n() > kMaxNCWidth) { err = "non-Clifford fragment too wide"; return CCS_ERR_NC_TOO_WIDE; }
    if (f.clifford && f.n() > kMaxBodyQubits) { err = "Clifford fragment too wide"; return CCS_ERR_UNSUPPORTED; }
    if (f.n_meas() > kMaxMeas) { err = "fragment measures too many wires"; return CCS_ERR_UNSUPPORTED; }
    p.frag_ids.push_back(fi);
  }
  // star: one fragment on every cut
  const int nf = (int)out.size() - first;
  if (nf > kMaxProblemFragments) {
    err = "more than " + std::to_string(kMaxProblemFragments) + " fragments in one problem";
    return CCS_ERR_UNSUPPORTED;
  }
  p.hub = -1;
  if (p.cuts.empty()) {
    p.hub = 0;
  } else {
    for (int h = 0; h < nf && p.hub < 0; ++h)
      if ((int)out[first + h].slots.size() == (int)p.cuts.size()) p.hub = h;
  }
  return CCS_OK;
}

namespace {
// Scratch of one host thread, kept between fragments and plan builds (the
// pool's threads persist), so compiling does not fault in fresh pages.
template <class Op>
struct CompileScratch {
  std::vector<Op> ops;
  std::vector<int> order, start;
  void reset(size_t gates) {
    ops.clear();
    ops.reserve(gates);                        // no reallocation while ops point at each other
  }
};
}  // namespace

void compile_clifford(Frag& f) {
  thread_local CompileScratch<PlaneOp> cs;
  cs.reset(f.gates.size());
  fuse_and_layer(f, cs.ops, cs.order, cs.start);
  const int nl = (int)cs.start.size() - 1;
  f.cops.clear();
  f.cops.reserve(cs.order.size());
  f.moment_start.assign(1, 0);
  f.moment_start.reserve(nl + 1);
  const uint16_t dummy = (uint16_t)f.n();
  for (int L = 0; L < nl; ++L) {
    for (int k = cs.start[L]; k < cs.start[L + 1]; ++k) {
      const PlaneOp& F = cs.ops[cs.order[k]];
      CliffordOp op = clifford_from_planes(F.px, F.pz, F.pf);
      op.qa = (uint16_t)F.a;
      op.qb = F.b >= 0 ? (uint16_t)F.b : dummy;
      f.cops.push_back(op);
    }
    f.moment_start.push_back((int)f.cops.size());
  }
}

void compile_nc(Frag& f) {
  thread_local CompileScratch<WordOp> cs;
  cs.reset(f.gates.size());
  fuse_and_layer(f, cs.ops, cs.order, cs.start);
  const int nl = (int)cs.start.size() - 1;
  f.nops.clear();
  f.moment_start.assign(1, 0);
  for (int L = 0; L < nl; ++L) {
    for (int k = cs.start[L]; k < cs.start[L + 1]; ++k) {
      const WordOp* F = &cs.ops[cs.order[k]];
      NCOp o{};
      o.a = F->a;
      o.b = F->b;
      if (F->b < 0) {
        cd U[4] = {1, 0, 0, 1};    // U <- G U: rows 0 and 1 of the 2x2
        for (auto& g : F->word) mix_rows(g.op, g.param, U, U + 2, 2);
        for (int i = 0; i < 4; ++i) { o.m[2 * i] = (float)U[i].real(); o.m[2 * i + 1] = (float)U[i].imag(); }
      } else {
        // U <- G U gate by gate, as row operations on the 4x4 (index = bit_a + 2 bit_b)
        cd U[16];
        for (int i = 0; i < 16; ++i) U[i] = (i % 5 == 0) ? 1.0 : 0.0;
        for (auto& g : F->word) {
          const int op = g.op, ra = g.ra, rb = g.rb < 0 ? 1 - g.ra : g.rb;
          if (op == CCS_CX) {          // rows with control bit set: swap the target bit
            for (int i = 0; i < 4; ++i)
              if (((i >> ra) & 1) && !((i >> rb) & 1))
                for (int j = 0; j < 4; ++j) std::swap(U[i * 4 + j], U[(i | (1 << rb)) * 4 + j]);
          } else if (op == CCS_CZ) {   // row with both bits set: negate
            for (int j = 0; j < 4; ++j) U[3 * 4 + j] = -U[3 * 4 + j];
          } else {                     // one-qubit gate on role ra: mix row pairs
            for (int i0 = 0; i0 < 4; ++i0) {
              if ((i0 >> ra) & 1) continue;
              mix_rows(op, g.param, U + i0 * 4, U + (i0 | (1 << ra)) * 4, 4);
            }
          }
        }
        for (int i = 0; i < 16; ++i) { o.m[2 * i] = (float)U[i].real(); o.m[2 * i + 1] = (float)U[i].imag(); }
      }
      f.nops.push_back(o);
    }
    f.moment_start.push_back((int)f.nops.size());
  }
}

static const std::vector<std::vector<int>> kPrepWords = {{}, {CCS_X}, {CCS_H}, {CCS_H, CCS_S}};
static const std::vector<std::vector<int>> kBasisWords = {{CCS_H}, {CCS_SDG, CCS_H}, {}};

static CliffordOp one_qubit_op(const std::vector<int>& w) {
  std::vector<std::array<int, 3>> word;
  for (int g : w) word.push_back({g, 0, -1});
  return clifford_from_word(word);
}

CliffordOp prep_op(int s) { return one_qubit_op(kPrepWords[s]); }
CliffordOp basis_op(int b) { return one_qubit_op(kBasisWords[b]); }

static void one_qubit_matrix(const std::vector<int>& w, float out[8]) {
  cd U[4] = {1, 0, 0, 1};
  for (int g : w) {
    cd G[4], R[4];
    gate_matrix_1q(g, 0.0, G);
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) R[i * 2 + j] = G[i * 2] * U[j] + G[i * 2 + 1] * U[2 + j];
    for (int i = 0; i < 4; ++i) U[i] = R[i];
  }
  for (int i = 0; i < 4; ++i) { out[2 * i] = (float)U[i].real(); out[2 * i + 1] = (float)U[i].imag(); }
}

void prep_matrix(int s, float out[8]) { one_qubit_matrix(kPrepWords[s], out); }
void basis_matrix(int b, float out[8]) { one_qubit_matrix(kBasisWords[b], out); }

}  // namespace ccs
