// Greedy cut search (Sec. V-A): the cutter tags non-Clifford operations and
// places wire cuts that isolate them into small non-Clifford fragments, the
// rest of the circuit staying Clifford.  The paper gives no search algorithm;
// this one grows regions from the non-Clifford gates:
//
//   * a region is a set of wire windows (qubit q, gate positions [a, b) of
//     q's gate list); its gates are those inside every window they touch, and
//     it is closed: a two-qubit gate inside one window is inside its partner's
//     window too;
//   * each window costs a cut before it (a > 0) and after it (b < len);
//     windows absorb runs of one-qubit gates at their edges;
//   * every non-Clifford gate seeds a one-gate window; overlapping regions
//     are merged;
//   * moves: widen a window by one gate, widen it to the start or end of its
//     wire or to the whole wire, saturate a region (make its windows whole
//     wires while the closure fits the width cap), or merge two regions (each followed by
//     closure); a beam of the cheapest states by estimated cost is expanded
//     (uphill moves allowed) until the best valid candidate stops improving;
//   * cost = sum over fragments of variants x per-variant work + 4^k 2^|o|
//     recombination work, with region width capped at max_nc_width.
// Every visited state that is a valid star (one Clifford fragment on every
// cut) within the cut budget is kept as a candidate, cheapest first.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <set>

#include "plan.hpp"

namespace ccs {

namespace {

struct Window {
  int q, a, b;
  // positions [sa, sb) already closed: every two-qubit gate there has its
  // partner position inside the region (empty when sa == sb).  Windows only
  // grow, so a closed position stays closed.
  int sa = 0, sb = 0;
};
using Region = std::vector<Window>;   // sorted by qubit, one window per qubit

struct Ctx {
  const Problem* P;
  int n;
  std::vector<std::vector<int>> ops_on;      // gate indices per qubit
  std::vector<std::vector<int>> tq_before;   // per qubit: two-qubit gates among ops_on[q][0, pos)
  std::vector<std::array<int, 2>> pos_of;    // position of gate g in ops_on[q0], ops_on[q1]
  std::vector<int> nonclifford;
  std::vector<char> in_marginal;
};

bool two_qubit(int op) { return op == CCS_CX || op == CCS_CZ; }

Window* find_w(Region& r, int q) {
  for (auto& w : r)
    if (w.q == q) return &w;
  return nullptr;
}

// Close a region under two-qubit gates.  Windows also absorb the runs of
// one-qubit gates at their edges: that pulls in no new qubit and lets a
// window reach the end of its wire, which removes a cut.
void close_region(const Ctx& C, Region& r) {
  bool changed = true;
  while (changed) {
    changed = false;
    for (auto& w : r) {
      const auto& ops = C.ops_on[w.q];
      while (w.a > 0 && !two_qubit(C.P->gates[ops[w.a - 1]][0])) --w.a;
      while (w.b < (int)ops.size() && !two_qubit(C.P->gates[ops[w.b]][0])) ++w.b;
    }
    for (size_t i = 0; i < r.size(); ++i) {
      const Window w = r[i];
      const int q = w.q;
      auto scan = [&](int lo, int hi) {
        for (int pos = lo; pos < hi; ++pos) {
          const int g = C.ops_on[q][pos];
          const auto& G = C.P->gates[g];
          if (!two_qubit(G[0])) continue;
          const int p = G[1] == q ? G[2] : G[1];
          const int pp = C.pos_of[g][G[1] == q ? 1 : 0];
          Window* o = find_w(r, p);
          if (!o) {
            r.push_back({p, pp, pp + 1});
            changed = true;
          } else if (pp < o->a || pp >= o->b) {
            o->a = std::min(o->a, pp);
            o->b = std::max(o->b, pp + 1);
            changed = true;
          }
        }
      };
      if (w.sa == w.sb) {
        scan(w.a, w.b);
      } else {
        scan(w.a, w.sa);
        scan(w.sb, w.b);
      }
      r[i].sa = w.a;
      r[i].sb = w.b;
    }
  }
  std::sort(r.begin(), r.end(), [](const Window& x, const Window& y) { return x.q < y.q; });
}

bool overlap(const Region& x, const Region& y) {
  for (auto& a : x)
    for (auto& b : y)
      if (a.q == b.q && a.a < b.b && b.a < a.b) return true;
  return false;
}

Region merge(const Region& x, const Region& y) {
  Region r = x;
  for (auto& w : y) {
    Window* o = find_w(r, w.q);
    if (!o) {
      r.push_back(w);
      continue;
    }
    o->a = std::min(o->a, w.a);
    o->b = std::max(o->b, w.b);
    // closed positions: the union when the two closed ranges meet, else the longer one
    if (w.sa == w.sb) continue;
    if (o->sa == o->sb || (std::max(o->sa, w.sa) <= std::min(o->sb, w.sb))) {
      const bool oe = o->sa == o->sb;
      o->sa = oe ? w.sa : std::min(o->sa, w.sa);
      o->sb = oe ? w.sb : std::max(o->sb, w.sb);
    } else if (w.sb - w.sa > o->sb - o->sa) {
      o->sa = w.sa;
      o->sb = w.sb;
    }
  }
  return r;
}

// Merge overlapping regions and re-close until stable.
void normalise(const Ctx& C, std::vector<Region>& rs) {
  for (auto& r : rs) close_region(C, r);
  bool changed = true;
  while (changed) {
    changed = false;
    for (size_t i = 0; i < rs.size() && !changed; ++i)
      for (size_t j = i + 1; j < rs.size() && !changed; ++j)
        if (overlap(rs[i], rs[j])) {
          rs[i] = merge(rs[i], rs[j]);
          close_region(C, rs[i]);
          rs.erase(rs.begin() + j);
          changed = true;
        }
  }
  std::sort(rs.begin(), rs.end(), [](const Region& x, const Region& y) {
    return std::make_pair(x[0].q, x[0].a) < std::make_pair(y[0].q, y[0].a);
  });
}

// Make windows whole wires one at a time, keeping each change whose closure
// still fits the width cap, until nothing changes.
Region saturate(const Ctx& C, Region r, int max_width) {
  bool changed = true;
  while (changed) {
    changed = false;
    for (size_t i = 0; i < r.size(); ++i) {
      const int len = (int)C.ops_on[r[i].q].size();
      if (r[i].a == 0 && r[i].b == len) continue;
      Region t = r;
      t[i].a = 0;
      t[i].b = len;
      close_region(C, t);
      if ((int)t.size() <= max_width) {
        r = t;
        changed = true;
        break;
      }
    }
  }
  return r;
}

std::vector<ccs_cut> cuts_of(const Ctx& C, const std::vector<Region>& rs) {
  std::vector<ccs_cut> cuts;
  for (auto& r : rs)
    for (auto& w : r) {
      const int len = (int)C.ops_on[w.q].size();
      if (w.a > 0) cuts.push_back({(uint32_t)w.q, (uint32_t)C.ops_on[w.q][w.a]});
      if (w.b < len) cuts.push_back({(uint32_t)w.q, (uint32_t)C.ops_on[w.q][w.b]});
    }
  std::sort(cuts.begin(), cuts.end(), [](const ccs_cut& x, const ccs_cut& y) {
    return x.gate_index != y.gate_index ? x.gate_index < y.gate_index : x.qubit < y.qubit;
  });
  cuts.erase(std::unique(cuts.begin(), cuts.end(), [](const ccs_cut& x, const ccs_cut& y) {
               return x.qubit == y.qubit && x.gate_index == y.gate_index;
             }), cuts.end());
  return cuts;
}

// Estimated work of a state straight from its windows (the Clifford rest is
// taken as one fragment).
// (The regions are closed: a two-qubit gate inside one window is inside its
// partner's window too, so the region's distinct gates are the window
// lengths less half the two-qubit positions.)
double estimate(const Ctx& C, const std::vector<Region>& rs, int max_width, bool* ok) {
  *ok = true;
  const int n = C.n;
  long long nc_gates_total = 0;
  double cost = 0.0;
  int k = 0, body_qin = 0, body_qout = 0, body_wires = n, body_marg = 0, nc_marg = 0;
  for (auto& r : rs) {
    int width = (int)r.size(), qin = 0, qout = 0;
    long long len_sum = 0, tq_sum = 0;
    for (auto& w : r) {
      len_sum += w.b - w.a;
      tq_sum += C.tq_before[w.q][w.b] - C.tq_before[w.q][w.a];
    }
    const long long gates = len_sum - tq_sum / 2;
    for (auto& w : r) {
      const int len = (int)C.ops_on[w.q].size();
      const bool pre = w.a > 0, post = w.b < len;
      qin += pre;
      qout += post;
      body_wires += (pre && post) ? 1 : (!pre && !post) ? -1 : 0;
      if (!post && C.in_marginal[w.q]) ++nc_marg;
    }
    if (width > max_width) *ok = false;
    k += qin + qout;
    body_qin += qout;
    body_qout += qin;
    nc_gates_total += gates;
    cost += std::pow(4.0, qin) * std::pow(3.0, qout) * (double)gates * std::ldexp(1.0, width) / 64.0;
  }
  body_marg = (int)C.P->marginal.size() - nc_marg;
  const long long body_gates = (long long)C.P->gates.size() - nc_gates_total;
  const double W = 2.0 * std::ceil(std::max(1, body_wires) / 64.0);
  cost += std::pow(4.0, body_qin) * std::pow(3.0, body_qout) * ((double)body_gates / 6.0 * W + 1024.0);
  cost += std::pow(4.0, k) * std::ldexp(1.0, body_marg + nc_marg) / 16.0;
  (void)body_marg;
  return cost;
}

}  // namespace

// The fragments a cut set gives, counted without building them: the same
// segments, union-find and checks as fragment_problem, keeping per fragment
// only its wire, gate, input/output and marginal counts.  Fragments are
// numbered by their first segment, as fragment_problem orders them, so the
// cost sums in the same order.
double plan_cost(const Problem& p, const std::vector<ccs_cut>& cuts_in, bool* ok) {
  auto invalid = [&]() {
    if (ok) *ok = false;
    return (double)INFINITY;
  };
  const int n = (int)p.n_qubits;
  const int ng = (int)p.gates.size();
  std::vector<ccs_cut> cuts = cuts_in;
  for (auto& c : cuts)
    if ((int)c.qubit >= n || (int)c.gate_index > ng) return invalid();
  std::sort(cuts.begin(), cuts.end(), [](const ccs_cut& x, const ccs_cut& y) {
    return x.gate_index != y.gate_index ? x.gate_index < y.gate_index : x.qubit < y.qubit;
  });
  for (size_t i = 1; i < cuts.size(); ++i)
    if (cuts[i].qubit == cuts[i - 1].qubit && cuts[i].gate_index == cuts[i - 1].gate_index) return invalid();
  if ((int)cuts.size() > kMaxCuts || p.marginal.size() > (size_t)kMaxMarginal) return invalid();
  for (size_t i = 0; i < p.marginal.size(); ++i) {
    if ((int)p.marginal[i] >= n) return invalid();
    for (size_t j = 0; j < i; ++j)
      if (p.marginal[i] == p.marginal[j]) return invalid();
  }
  // cut positions per qubit, ascending (cuts are sorted by gate index)
  std::vector<int> cnt(n + 1, 0), start(n + 1, 0), pos(cuts.size());
  for (auto& c : cuts) cnt[c.qubit]++;
  for (int q = 0; q < n; ++q) start[q + 1] = start[q] + cnt[q];
  {
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (auto& c : cuts) pos[fill[c.qubit]++] = (int)c.gate_index;
  }
  std::vector<int> base(n + 1, 0);
  for (int q = 0; q < n; ++q) base[q + 1] = base[q] + cnt[q] + 1;
  // one pass over the gates: each qubit's current segment follows a cursor
  // over the cuts (sorted by gate index); two-qubit gates join segments, and
  // every segment counts its gates (a gate belongs to its first operand's)
  // and whether one of them is non-Clifford
  UF uf(base[n]);
  std::vector<int> seg_gates(base[n], 0), segcur(base.begin(), base.end() - 1);
  std::vector<char> seg_nc(base[n], 0);
  {
    size_t nc = 0;
    for (int gi = 0; gi < ng; ++gi) {
      while (nc < cuts.size() && (int)cuts[nc].gate_index <= gi) ++segcur[cuts[nc++].qubit];
      const auto& g = p.gates[gi];
      const int sa = segcur[g[1]];
      ++seg_gates[sa];
      if (two_qubit(g[0])) uf.join(sa, segcur[g[2]]);
      else if (is_nonclifford_op(g[0])) seg_nc[sa] = 1;
    }
  }
  std::vector<int> fid(base[n], -1), of_seg(base[n]);
  int nf = 0;
  for (int s = 0; s < base[n]; ++s) {
    const int r = uf.find(s);
    if (fid[r] < 0) fid[r] = nf++;
    of_seg[s] = fid[r];
  }
  std::vector<int> wires(nf, 0), gates(nf, 0), qin(nf, 0), qout(nf, 0), marg(nf, 0);
  std::vector<char> cliff(nf, 1);
  for (int s = 0; s < base[n]; ++s) {
    wires[of_seg[s]]++;
    gates[of_seg[s]] += seg_gates[s];
    if (seg_nc[s]) cliff[of_seg[s]] = 0;
  }
  for (auto& c : cuts) {
    const int q = (int)c.qubit;
    const int k = (int)(std::find(pos.begin() + start[q], pos.begin() + start[q] + cnt[q], (int)c.gate_index) -
                        (pos.begin() + start[q])) + 1;
    const int fu = of_seg[base[q] + k - 1], fd = of_seg[base[q] + k];
    if (fu == fd) return invalid();
    qout[fu]++;
    qin[fd]++;
  }
  for (auto q : p.marginal) marg[of_seg[base[q] + cnt[q]]]++;
  bool star = cuts.empty();
  for (int f = 0; f < nf; ++f) {
    if (!cliff[f] && wires[f] > kMaxNCWidth) return invalid();
    if (cliff[f] && wires[f] > kMaxBodyQubits) return invalid();
    if (marg[f] + qout[f] > kMaxMeas) return invalid();
    if (qin[f] + qout[f] == (int)cuts.size()) star = true;
  }
  if (!star) return invalid();
  double cost = 0.0;
  for (int f = 0; f < nf; ++f) {
    int v = 1;
    for (int i = 0; i < qin[f]; ++i) v *= 4;
    for (int i = 0; i < qout[f]; ++i) v *= 3;
    const double nv = (double)v;
    if (cliff[f]) cost += nv * ((double)gates[f] / 6.0 * 2.0 * std::ceil(wires[f] / 64.0) + 1024.0);
    else cost += nv * (double)gates[f] * std::ldexp(1.0, wires[f]) / 64.0;
  }
  cost += std::pow(4.0, (double)cuts.size()) * std::ldexp(1.0, (int)p.marginal.size()) / 16.0;
  if (ok) *ok = true;
  return cost;
}

int greedy_cuts(const Problem& p, const CutSearchOpts& o, std::vector<CutCandidate>& cands, std::string& err) {
  Ctx C;
  C.P = &p;
  C.n = (int)p.n_qubits;
  C.ops_on.assign(C.n, {});
  C.pos_of.assign(p.gates.size(), {-1, -1});
  for (int g = 0; g < (int)p.gates.size(); ++g) {
    const auto& G = p.gates[g];
    if (G[1] < 0 || G[1] >= C.n || (two_qubit(G[0]) && (G[2] < 0 || G[2] >= C.n))) {
      err = "gate qubit out of range";
      return CCS_ERR_INVALID_ARG;
    }
    C.pos_of[g][0] = (int)C.ops_on[G[1]].size();
    C.ops_on[G[1]].push_back(g);
    if (two_qubit(G[0])) {
      C.pos_of[g][1] = (int)C.ops_on[G[2]].size();
      C.ops_on[G[2]].push_back(g);
    }
    if (is_nonclifford_op(G[0])) C.nonclifford.push_back(g);
  }
  C.tq_before.assign(C.n, {});
  for (int q = 0; q < C.n; ++q) {
    auto& t = C.tq_before[q];
    t.assign(C.ops_on[q].size() + 1, 0);
    for (size_t i = 0; i < C.ops_on[q].size(); ++i) t[i + 1] = t[i] + (two_qubit(p.gates[C.ops_on[q][i]][0]) ? 1 : 0);
  }
  C.in_marginal.assign(C.n, 0);
  for (auto q : p.marginal)
    if ((int)q < C.n) C.in_marginal[q] = 1;
  cands.clear();
  if (C.nonclifford.empty()) {
    cands.push_back({{}, 0.0, {}});
    return CCS_OK;
  }
  std::vector<Region> state;
  for (int g : C.nonclifford) {
    const int q = p.gates[g][1];
    state.push_back({{q, C.pos_of[g][0], C.pos_of[g][0] + 1}});
  }
  normalise(C, state);
  std::map<std::vector<std::pair<int, int>>, double> seen;
  auto key_of = [&](const std::vector<Region>& s) {
    std::vector<std::pair<int, int>> key;
    for (auto& r : s) {
      for (auto& w : r) key.push_back({w.q * 4 + 0, w.a}), key.push_back({w.q * 4 + 1, w.b});
      key.push_back({-1, -1});
    }
    return key;
  };
  std::set<std::vector<std::pair<int, int>>> cut_seen;
  auto record = [&](const std::vector<Region>& s) {
    for (auto& r : s)
      if ((int)r.size() > o.max_nc_width) return;
    auto cuts = cuts_of(C, s);
    if ((int)cuts.size() > o.max_cuts) return;
    std::vector<std::pair<int, int>> key;
    for (auto& c : cuts) key.push_back({(int)c.qubit, (int)c.gate_index});
    if (!cut_seen.insert(key).second) return;
    bool valid;
    const double cost = plan_cost(p, cuts, &valid);
    if (valid) cands.push_back({cuts, cost, {}});
  };
  // Beam search over region states (uphill moves allowed, so closures that
  // first add cuts and then remove them are found).
  struct Item { double cost; std::vector<Region> s; };
  const int beam = 6;
  bool ok;
  std::vector<Item> frontier{{estimate(C, state, o.max_nc_width, &ok), state}};
  record(state);
  double best_valid = INFINITY;
  int stale = 0;
  for (int iter = 0; iter < 2 * C.n + 64 && stale < 12; ++iter) {
    std::vector<Item> next;
    std::set<std::vector<std::pair<int, int>>> in_next;
    auto consider = [&](std::vector<Region> s) {
      normalise(C, s);
      bool ok2;
      const double c2 = estimate(C, s, o.max_nc_width, &ok2);
      if (!ok2) return;
      auto key = key_of(s);
      if (seen.count(key)) return;
      seen[key] = c2;
      if (!in_next.insert(key).second) return;
      next.push_back({c2, std::move(s)});
    };
    for (auto& it : frontier) {
      const auto& st = it.s;
      for (size_t ri = 0; ri < st.size(); ++ri) {
        for (size_t wi = 0; wi < st[ri].size(); ++wi) {
          const Window w = st[ri][wi];
          const int len = (int)C.ops_on[w.q].size();
          if (w.a > 0) {
            auto s1 = st; s1[ri][wi].a = w.a - 1; consider(s1);
            if (w.a > 1) { auto s2 = st; s2[ri][wi].a = 0; consider(s2); }
          }
          if (w.b < len) {
            auto s1 = st; s1[ri][wi].b = w.b + 1; consider(s1);
            if (w.b < len - 1) { auto s2 = st; s2[ri][wi].b = len; consider(s2); }
          }
          if (w.a > 0 && w.b < len) { auto s3 = st; s3[ri][wi].a = 0; s3[ri][wi].b = len; consider(s3); }
        }
        {
          auto s5 = st;
          s5[ri] = saturate(C, s5[ri], o.max_nc_width);
          consider(s5);
        }
        for (size_t rj = ri + 1; rj < st.size(); ++rj) {
          auto s4 = st;
          s4[ri] = merge(s4[ri], s4[rj]);
          s4.erase(s4.begin() + rj);
          consider(s4);
        }
      }
    }
    if (next.empty()) break;
    std::stable_sort(next.begin(), next.end(), [](const Item& x, const Item& y) { return x.cost < y.cost; });
    if (std::getenv("CCS_DEBUG_CUTTER")) {
      const auto& b = next.front();
      std::fprintf(stderr, "iter %d: %zu states, best est %.3g, regions %zu, cuts %zu, widths:", iter, next.size(),
                   b.cost, b.s.size(), cuts_of(C, b.s).size());
      for (auto& r : b.s) std::fprintf(stderr, " %zu", r.size());
      std::fprintf(stderr, "\n");
    }
    if ((int)next.size() > beam) next.resize(beam);
    for (auto& it : next) record(it.s);
    double bv = INFINITY;
    for (auto& c : cands) bv = std::min(bv, c.cost);
    if (bv < best_valid) { best_valid = bv; stale = 0; } else { ++stale; }
    frontier.swap(next);
  }
  if (cands.empty()) {
    err = "no valid cut set within the cut and width limits";
    return CCS_ERR_TOO_MANY_CUTS;
  }
  std::stable_sort(cands.begin(), cands.end(),
                   [](const CutCandidate& x, const CutCandidate& y) { return x.cost < y.cost; });
  return CCS_OK;
}

}  // namespace ccs
