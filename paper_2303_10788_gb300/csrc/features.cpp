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

#include "plan.hpp"

namespace ccs {

// Candidate-independent part: the interaction graph (CSR of A = D^-1 Adj and
// of the transposed values) and the per-qubit gate counts.
GraphBase graph_base(const Problem& p) {
  GraphBase g;
  const int n = (int)p.n_qubits;
  g.tcount.assign(n, 0);
  g.gcount.assign(n, 0);
  std::vector<std::pair<int, int>> e;
  for (auto& gt : p.gates) {
    g.gcount[gt[1]]++;
    if (is_nonclifford_op(gt[0])) g.tcount[gt[1]]++;
    if (gt[0] == CCS_CX || gt[0] == CCS_CZ) {
      g.gcount[gt[2]]++;
      e.push_back({gt[1], gt[2]});
      e.push_back({gt[2], gt[1]});
    }
  }
  std::sort(e.begin(), e.end());
  g.rowptr.assign(n + 1, 0);
  std::vector<int> w;                      // edge weights (gate counts), CSR order
  for (size_t i = 0; i < e.size();) {
    size_t j = i + 1;
    while (j < e.size() && e[j] == e[i]) ++j;
    g.col.push_back(e[i].second);
    w.push_back((int)(j - i));
    g.rowptr[e[i].first + 1]++;
    i = j;
  }
  for (int q = 0; q < n; ++q) g.rowptr[q + 1] += g.rowptr[q];
  std::vector<double> deg(n, 0.0);
  for (int q = 0; q < n; ++q)
    for (int t = g.rowptr[q]; t < g.rowptr[q + 1]; ++t) deg[q] += w[t];
  g.val.resize(w.size());
  g.val_t.resize(w.size());
  for (int q = 0; q < n; ++q)
    for (int t = g.rowptr[q]; t < g.rowptr[q + 1]; ++t) {
      g.val[t] = (float)(w[t] / deg[q]);
      g.val_t[t] = (float)(w[t] / deg[g.col[t]]);
    }
  return g;
}

// Candidate-dependent part: fragment the circuit under the cut set, then the
// node features (8 per qubit) and the global features.
int featurize_nodes(const Problem& p0, const GraphBase& g, const std::vector<ccs_cut>& cuts, std::vector<float>& x,
                    std::vector<float>& glob, std::string& err) {
  Problem p = p0;
  p.cuts = cuts;
  p.zstrings.clear();
  std::vector<Frag> frags;
  int rc = fragment_problem(p, 0, frags, err);
  if (rc != CCS_OK) return rc;
  const int n = (int)p.n_qubits;
  std::vector<int> nc_gates(n, 0), ncut(n, 0), marg(n, 0), in_hub(n, 0);
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
      for (auto& gt : f.gates) {
        per[gt[1]]++;
        if (gt[2] >= 0) per[gt[2]]++;
      }
      for (int li = 0; li < f.n(); ++li) nc_gates[f.wires[li].first] += per[li];
    }
    if (hub)
      for (auto& wr : f.wires) {
        const int q = (int)wr.first;
        if ((int)wr.second == ncut[q]) in_hub[q] = 1;     // the qubit's last segment
      }
  }
  x.assign((size_t)n * 8, 0.f);
  for (int q = 0; q < n; ++q) {
    float* r = &x[(size_t)q * 8];
    r[0] = 1.f;
    r[1] = g.tcount[q] / 4.f;
    r[2] = (g.rowptr[q + 1] - g.rowptr[q]) / 4.f;
    r[3] = g.gcount[q] / 100.f;
    r[4] = g.gcount[q] ? (float)nc_gates[q] / (float)g.gcount[q] : 0.f;
    r[5] = (float)ncut[q];
    r[6] = (float)marg[q];
    r[7] = (float)in_hub[q];
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

int featurize(const Problem& p0, const std::vector<ccs_cut>& cuts, std::vector<float>& x, std::vector<int>& rowptr,
              std::vector<int>& col, std::vector<float>& val, std::vector<float>& val_t, std::vector<float>& glob,
              std::string& err) {
  GraphBase g = graph_base(p0);
  int rc = featurize_nodes(p0, g, cuts, x, glob, err);
  if (rc != CCS_OK) return rc;
  rowptr = std::move(g.rowptr);
  col = std::move(g.col);
  val = std::move(g.val);
  val_t = std::move(g.val_t);
  return CCS_OK;
}

}  // namespace ccs
