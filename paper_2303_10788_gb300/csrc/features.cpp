// Graph features of one circuit under one candidate cut set, the input of the
// learned cut scorer: nodes are qubits, edges the two-qubit interactions
// (weight = gate count), A = D^-1 Adj.
//
// Node features (8): 1, T gates on the qubit / 4, distinct neighbours / 4,
// gates on the qubit / 100, fraction of the qubit's gates in non-Clifford
// fragments, cuts on the qubit, marginal qubit, final segment in the hub.
// Global features (8): cuts / 8, log2(hub variants) / 16,
// log2(non-hub variants) / 8, log2(4^k 2^|o|) / 24, widest non-Clifford
// fragment / 12, log2(n) / 9, log2(gates) / 17, fragments / 8.
#include <algorithm>
#include <cmath>
#include <map>

#include "plan.hpp"

namespace ccs {

int featurize(const Problem& p0, const std::vector<ccs_cut>& cuts, std::vector<float>& x, std::vector<int>& rowptr,
              std::vector<int>& col, std::vector<float>& val, std::vector<float>& val_t, std::vector<float>& glob,
              std::string& err) {
  Problem p = p0;
  p.cuts = cuts;
  p.zstrings.clear();
  std::vector<Frag> frags;
  int rc = fragment_problem(p, 0, frags, err);
  if (rc != CCS_OK) return rc;
  const int n = (int)p.n_qubits;
  std::vector<std::map<int, int>> adj(n);
  std::vector<int> tcount(n, 0), gcount(n, 0), nc_gates(n, 0), ncut(n, 0), marg(n, 0), in_hub(n, 0);
  for (auto& g : p.gates) {
    gcount[g[1]]++;
    if (is_nonclifford_op(g[0])) tcount[g[1]]++;
    if (g[0] == CCS_CX || g[0] == CCS_CZ) {
      gcount[g[2]]++;
      adj[g[1]][g[2]]++;
      adj[g[2]][g[1]]++;
    }
  }
  for (auto& c : p.cuts) ncut[c.qubit]++;
  for (auto q : p.marginal) marg[q] = 1;
  double hub_v = 1.0, other_v = 0.0;
  int max_nc = 0;
  for (int fi = 0; fi < (int)frags.size(); ++fi) {
    const Frag& f = frags[fi];
    const bool hub = fi == p.hub;
    if (hub) hub_v = (double)f.n_variants();
    else other_v += (double)f.n_variants();
    if (!f.clifford) max_nc = std::max(max_nc, f.n());
    // per-wire gate counts of non-Clifford fragments
    if (!f.clifford) {
      std::vector<int> per(f.n(), 0);
      for (auto& g : f.gates) {
        per[g[1]]++;
        if (g[2] >= 0) per[g[2]]++;
      }
      for (int li = 0; li < f.n(); ++li) nc_gates[f.wires[li].first] += per[li];
    }
    if (hub)
      for (auto& w : f.wires) {
        const int q = (int)w.first;
        int last = 0;
        for (auto& c : p.cuts)
          if ((int)c.qubit == q) ++last;
        if ((int)w.second == last) in_hub[q] = 1;
      }
  }
  x.assign((size_t)n * 8, 0.f);
  rowptr.assign(n + 1, 0);
  col.clear();
  val.clear();
  val_t.clear();
  std::vector<double> deg(n, 0.0);
  for (int q = 0; q < n; ++q)
    for (auto& e : adj[q]) deg[q] += e.second;
  for (int q = 0; q < n; ++q) {
    float* r = &x[(size_t)q * 8];
    r[0] = 1.f;
    r[1] = tcount[q] / 4.f;
    r[2] = adj[q].size() / 4.f;
    r[3] = gcount[q] / 100.f;
    r[4] = gcount[q] ? (float)nc_gates[q] / (float)gcount[q] : 0.f;
    r[5] = (float)ncut[q];
    r[6] = (float)marg[q];
    r[7] = (float)in_hub[q];
    for (auto& e : adj[q]) {
      col.push_back(e.first);
      val.push_back((float)(e.second / deg[q]));
      val_t.push_back((float)(e.second / deg[e.first]));
    }
    rowptr[q + 1] = (int)col.size();
  }
  const double k = (double)p.cuts.size();
  glob = {(float)(k / 8.0),
          (float)(std::log2(hub_v) / 16.0),
          (float)(std::log2(1.0 + other_v) / 8.0),
          (float)((2.0 * k + (double)p.marginal.size()) / 24.0),
          (float)(max_nc / 12.0),
          (float)(std::log2((double)n) / 9.0),
          (float)(std::log2(1.0 + (double)p.gates.size()) / 17.0),
          (float)(frags.size() / 8.0)};
  return CCS_OK;
}

}  // namespace ccs
