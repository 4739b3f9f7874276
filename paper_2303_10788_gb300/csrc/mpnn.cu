// Learned cut-set scorer: a message-passing network over the qubit
// interaction graph of a circuit with one candidate cut set applied, trained
// on measured evaluation + recombination times (its choices are judged by the
// greedy search's cost estimate, which remains the fallback).
//
//   h0      = relu(W_in x_v + b_in)                          (8 -> 64)
//   h_{l+1} = relu(Ws_l h_l + Wn_l (A h_l)_v + b_l)           l = 0, 1, 2
//   r_g     = mean_{v in g} h3_v
//   z_g     = relu(W_r1 [r_g, glob_g] + b_r1)                 (72 -> 64)
//   y_g     = w_r2 . z_g + b_r2                               predicted log time
//
// A is the degree-normalised adjacency (A = D^-1 Adj).  Weights are used in
// FP16 (rounded from an FP32 master copy that Adam updates); activations,
// gradients and accumulations are FP32.  Every step is a kernel below.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "abi_guard.hpp"
#include "kernels.cuh"

namespace ccs {
namespace mp {

constexpr int kIn = 8, kGlob = 8, kH = 64, kLayers = 3, kR = kH + kGlob;

// flat parameter layout
constexpr int oWin = 0, oBin = oWin + kH * kIn;
constexpr int oLayer = oBin + kH;
constexpr int kLayerSize = 2 * kH * kH + kH;   // Ws, Wn, b
constexpr int oWr1 = oLayer + kLayers * kLayerSize, oBr1 = oWr1 + kH * kR;
constexpr int oWr2 = oBr1 + kH, oBr2 = oWr2 + kH;
constexpr int kParams = oBr2 + 1;

// Y[r][o] = act(sum_i X1[r][i] W1[o][i] + sum_j X2[r][j] W2[o][j] + b[o]),
// weights in FP16; one thread per (row, output).
__global__ void dense_fwd(const float* X1, int d1, const half* W1, const float* X2, const half* W2,
                          const half* b, int rows, int relu, float* Y) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)rows * kH) return;
  const int r = (int)(t / kH), o = (int)(t % kH);
  float acc = __half2float(b[o]);
  for (int i = 0; i < d1; ++i) acc = fmaf(X1[(long long)r * d1 + i], __half2float(W1[o * d1 + i]), acc);
  if (X2)
    for (int j = 0; j < kH; ++j) acc = fmaf(X2[(long long)r * kH + j], __half2float(W2[o * kH + j]), acc);
  Y[t] = relu ? fmaxf(acc, 0.f) : acc;
}

// Y = A X over CSR rows (X, Y: rows x 64)
__global__ void spmm(const int* rowptr, const int* col, const float* val, const float* X, int rows, float* Y) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)rows * kH) return;
  const int r = (int)(t / kH), c = (int)(t % kH);
  float acc = 0.f;
  for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) acc = fmaf(val[e], X[(long long)col[e] * kH + c], acc);
  Y[t] = acc;
}

// R[g][c] = mean over the graph's nodes; the global features follow in [64, 72)
__global__ void seg_mean_cat(const int* goff, const float* H, const float* glob, int graphs, float* RG) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= graphs * kR) return;
  const int g = t / kR, c = t % kR;
  if (c >= kH) {
    RG[t] = glob[g * kGlob + (c - kH)];
    return;
  }
  const int a = goff[g], b = goff[g + 1];
  float acc = 0.f;
  for (int v = a; v < b; ++v) acc += H[(long long)v * kH + c];
  RG[t] = b > a ? acc / (float)(b - a) : 0.f;
}

__global__ void head_fwd(const float* Z, const half* w2, const half* b2, int graphs, float* y) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= graphs) return;
  float acc = __half2float(b2[0]);
  for (int j = 0; j < kH; ++j) acc = fmaf(Z[g * kH + j], __half2float(w2[j]), acc);
  y[g] = acc;
}

// --- backward -------------------------------------------------------------
// loss = mean_g (y_g - t_g)^2 ; dy, grads of the head, dZ (through relu)
__global__ void head_bwd(const float* y, const float* tgt, const float* Z, const half* w2, int graphs, float* loss,
                         float* dZ, float* grad) {
  // one block; graphs <= a few thousand
  __shared__ float red[256];
  float l = 0.f;
  for (int g = threadIdx.x; g < graphs; g += blockDim.x) {
    const float d = y[g] - tgt[g];
    l += d * d;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / graphs;
  for (int j = threadIdx.x; j <= kH; j += blockDim.x) {   // w_r2 (64) and b_r2
    float acc = 0.f;
    for (int g = 0; g < graphs; ++g) {
      const float dy = 2.f * (y[g] - tgt[g]) / graphs;
      acc += j < kH ? dy * Z[g * kH + j] : dy;
    }
    grad[oWr2 + j] = acc;   // oBr2 == oWr2 + kH
  }
  for (int t = threadIdx.x; t < graphs * kH; t += blockDim.x) {
    const int g = t / kH, j = t % kH;
    const float dy = 2.f * (y[g] - tgt[g]) / graphs;
    dZ[t] = Z[t] > 0.f ? dy * __half2float(w2[j]) : 0.f;
  }
}

// dW[o][i] += sum_r dP[r][o] X[r][i]  (and db[o] when i == d): one thread per (o, i)
__global__ void wgrad(const float* dP, const float* X, int d, int rows, float* dW, float* db) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kH * (d + 1)) return;
  const int o = t / (d + 1), i = t % (d + 1);
  float acc = 0.f;
  if (i < d)
    for (int r = 0; r < rows; ++r) acc = fmaf(dP[(long long)r * kH + o], X[(long long)r * d + i], acc);
  else
    for (int r = 0; r < rows; ++r) acc += dP[(long long)r * kH + o];
  if (i < d) dW[o * d + i] += acc;
  else if (db) db[o] += acc;
}

// dX[r][i] = sum_o dP[r][o] W[o][i]  (W: 64 x d, fp16), optionally += existing
__global__ void dgrad(const float* dP, const half* W, int d, int rows, int accumulate, float* dX) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)rows * d) return;
  const int r = (int)(t / d), i = (int)(t % d);
  float acc = 0.f;
  for (int o = 0; o < kH; ++o) acc = fmaf(dP[(long long)r * kH + o], __half2float(W[o * d + i]), acc);
  dX[t] = accumulate ? dX[t] + acc : acc;
}

__global__ void relu_mask(const float* H, float* dH, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n && !(H[t] > 0.f)) dH[t] = 0.f;
}

// dH3[v] = dR[g(v)] / n_g   (first 64 columns of d[R, G])
__global__ void seg_mean_bwd(const int* goff, const int* node_graph, const float* dRG, int nodes, float* dH) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nodes * kH) return;
  const int v = (int)(t / kH), c = (int)(t % kH);
  const int g = node_graph[v];
  dH[t] = dRG[g * kR + c] / (float)(goff[g + 1] - goff[g]);
}

__global__ void adam(float* master, half* w16, const float* grad, float* m, float* v, int n, float lr, float b1,
                     float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grad[i];
  m[i] = b1 * m[i] + (1.f - b1) * g;
  v[i] = b2 * v[i] + (1.f - b2) * g * g;
  master[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
  w16[i] = __float2half_rn(master[i]);
}

__global__ void to_half(const float* src, half* dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2half_rn(src[i]);
}

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace mp
}  // namespace ccs

using namespace ccs;
using namespace ccs::mp;

struct ccs_mpnn_s {
  ccs_ctx ctx;
  float* master = nullptr;   // FP32 master weights
  half* w16 = nullptr;       // FP16 weights used by the forward
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  long long step = 0;
};

namespace {

// device copies of one graph batch + activations
struct Batch {
  int n = 0, g = 0;
  int *rowptr = nullptr, *col = nullptr, *goff = nullptr, *ngraph = nullptr;
  float *val = nullptr, *valt = nullptr, *x = nullptr, *glob = nullptr, *tgt = nullptr;
  float* H[kLayers + 1] = {};
  float* AH[kLayers] = {};
  float *RG = nullptr, *Z = nullptr, *y = nullptr, *loss = nullptr, *dZ = nullptr, *dRG = nullptr;
  float *dH = nullptr, *dP = nullptr, *tmp = nullptr;
  std::vector<void*> all;
  cudaError_t err = cudaSuccess;
  template <class T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (p) all.push_back(p);
    return (T*)p;
  }
  ~Batch() {
    for (void* p : all) cudaFree(p);
  }
};

}  // namespace

// Host-side checks of a batch: every index the kernels follow stays in range.
static bool batch_ok(const ccs_graph_batch* b) {
  if (b->n_nodes < 0 || b->n_graphs <= 0 || !b->x || !b->rowptr || !b->graph_off || !b->glob) return false;
  if (b->rowptr[0] != 0 || b->graph_off[0] != 0 || b->graph_off[b->n_graphs] != b->n_nodes) return false;
  for (int g = 0; g < b->n_graphs; ++g)
    if (b->graph_off[g + 1] < b->graph_off[g]) return false;
  for (int v = 0; v < b->n_nodes; ++v)
    if (b->rowptr[v + 1] < b->rowptr[v]) return false;
  const int nnz = b->rowptr[b->n_nodes];
  if (nnz > 0 && (!b->col || !b->val || !b->val_t)) return false;
  for (int e = 0; e < nnz; ++e)
    if (b->col[e] < 0 || b->col[e] >= b->n_nodes) return false;
  return true;
}

static int upload_batch(const ccs_graph_batch* b, const float* target, cudaStream_t s, Batch& d) {
  if (!batch_ok(b)) return CCS_ERR_INVALID_ARG;
  d.n = b->n_nodes;
  d.g = b->n_graphs;
  const int nnz = b->rowptr[b->n_nodes];
  d.rowptr = d.alloc<int>(d.n + 1);
  d.col = d.alloc<int>(nnz);
  d.val = d.alloc<float>(nnz);
  d.valt = d.alloc<float>(nnz);
  d.goff = d.alloc<int>(d.g + 1);
  d.ngraph = d.alloc<int>(d.n);
  d.x = d.alloc<float>((size_t)d.n * kIn);
  d.glob = d.alloc<float>((size_t)d.g * kGlob);
  d.tgt = d.alloc<float>(d.g);
  for (int l = 0; l <= kLayers; ++l) d.H[l] = d.alloc<float>((size_t)d.n * kH);
  for (int l = 0; l < kLayers; ++l) d.AH[l] = d.alloc<float>((size_t)d.n * kH);
  d.RG = d.alloc<float>((size_t)d.g * kR);
  d.Z = d.alloc<float>((size_t)d.g * kH);
  d.y = d.alloc<float>(d.g);
  d.loss = d.alloc<float>(1);
  d.dZ = d.alloc<float>((size_t)d.g * kH);
  d.dRG = d.alloc<float>((size_t)d.g * kR);
  d.dH = d.alloc<float>((size_t)d.n * kH);
  d.dP = d.alloc<float>((size_t)d.n * kH);
  d.tmp = d.alloc<float>((size_t)d.n * kH);
  if (d.err != cudaSuccess) return CCS_ERR_OOM;
  std::vector<int> ng(d.n);
  for (int g = 0; g < d.g; ++g)
    for (int v = b->graph_off[g]; v < b->graph_off[g + 1]; ++v) ng[v] = g;
  cudaMemcpyAsync(d.rowptr, b->rowptr, (d.n + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d.col, b->col, nnz * sizeof(int), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d.val, b->val, nnz * sizeof(float), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d.valt, b->val_t, nnz * sizeof(float), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d.goff, b->graph_off, (d.g + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d.ngraph, ng.data(), d.n * sizeof(int), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d.x, b->x, (size_t)d.n * kIn * sizeof(float), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d.glob, b->glob, (size_t)d.g * kGlob * sizeof(float), cudaMemcpyHostToDevice, s);
  if (target) cudaMemcpyAsync(d.tgt, target, d.g * sizeof(float), cudaMemcpyHostToDevice, s);
  // the host vector must outlive the copy
  cudaStreamSynchronize(s);
  return cudaGetLastError() == cudaSuccess ? CCS_OK : CCS_ERR_CUDA;
}

static void forward(ccs_mpnn net, Batch& d, cudaStream_t s) {
  const half* W = net->w16;
  dense_fwd<<<blocks((long long)d.n * kH), 256, 0, s>>>(d.x, kIn, W + oWin, nullptr, nullptr, W + oBin, d.n, 1, d.H[0]); note_launch();
  for (int l = 0; l < kLayers; ++l) {
    const half* L = W + oLayer + l * kLayerSize;
    spmm<<<blocks((long long)d.n * kH), 256, 0, s>>>(d.rowptr, d.col, d.val, d.H[l], d.n, d.AH[l]); note_launch();
    dense_fwd<<<blocks((long long)d.n * kH), 256, 0, s>>>(d.H[l], kH, L, d.AH[l], L + kH * kH, L + 2 * kH * kH,
                                                          d.n, 1, d.H[l + 1]); note_launch();
  }
  seg_mean_cat<<<blocks((long long)d.g * kR), 256, 0, s>>>(d.goff, d.H[kLayers], d.glob, d.g, d.RG); note_launch();
  dense_fwd<<<blocks((long long)d.g * kH), 256, 0, s>>>(d.RG, kR, W + oWr1, nullptr, nullptr, W + oBr1, d.g, 1, d.Z); note_launch();
  head_fwd<<<blocks(d.g), 256, 0, s>>>(d.Z, W + oWr2, W + oBr2, d.g, d.y); note_launch();
}

static void backward(ccs_mpnn net, Batch& d, cudaStream_t s) {
  const half* W = net->w16;
  float* G = net->grad;
  cudaMemsetAsync(G, 0, kParams * sizeof(float), s);
  head_bwd<<<1, 256, 0, s>>>(d.y, d.tgt, d.Z, W + oWr2, d.g, d.loss, d.dZ, G); note_launch();
  wgrad<<<blocks(kH * (kR + 1)), 256, 0, s>>>(d.dZ, d.RG, kR, d.g, G + oWr1, G + oBr1); note_launch();
  dgrad<<<blocks((long long)d.g * kR), 256, 0, s>>>(d.dZ, W + oWr1, kR, d.g, 0, d.dRG); note_launch();
  seg_mean_bwd<<<blocks((long long)d.n * kH), 256, 0, s>>>(d.goff, d.ngraph, d.dRG, d.n, d.dH); note_launch();
  for (int l = kLayers - 1; l >= 0; --l) {
    const half* L = W + oLayer + l * kLayerSize;
    float* GL = G + oLayer + l * kLayerSize;
    cudaMemcpyAsync(d.dP, d.dH, (size_t)d.n * kH * sizeof(float), cudaMemcpyDeviceToDevice, s);
    relu_mask<<<blocks((long long)d.n * kH), 256, 0, s>>>(d.H[l + 1], d.dP, (long long)d.n * kH); note_launch();
    wgrad<<<blocks(kH * (kH + 1)), 256, 0, s>>>(d.dP, d.H[l], kH, d.n, GL, GL + 2 * kH * kH); note_launch();
    wgrad<<<blocks(kH * (kH + 1)), 256, 0, s>>>(d.dP, d.AH[l], kH, d.n, GL + kH * kH, nullptr); note_launch();
    // dH_l = dP Ws + A^T (dP Wn)
    dgrad<<<blocks((long long)d.n * kH), 256, 0, s>>>(d.dP, L + kH * kH, kH, d.n, 0, d.tmp); note_launch();
    spmm<<<blocks((long long)d.n * kH), 256, 0, s>>>(d.rowptr, d.col, d.valt, d.tmp, d.n, d.dH); note_launch();
    dgrad<<<blocks((long long)d.n * kH), 256, 0, s>>>(d.dP, L, kH, d.n, 1, d.dH); note_launch();
  }
  cudaMemcpyAsync(d.dP, d.dH, (size_t)d.n * kH * sizeof(float), cudaMemcpyDeviceToDevice, s);
  relu_mask<<<blocks((long long)d.n * kH), 256, 0, s>>>(d.H[0], d.dP, (long long)d.n * kH); note_launch();
  wgrad<<<blocks(kH * (kIn + 1)), 256, 0, s>>>(d.dP, d.x, kIn, d.n, G + oWin, G + oBin); note_launch();
}

extern "C" {

int ccs_mpnn_num_params(void) { return kParams; }

int ccs_mpnn_create(ccs_ctx c, uint64_t seed, ccs_mpnn* out) {
  return abi_guard([](int code, const char*) { return code; }, [&]() -> int {
    if (!c || !out) return CCS_ERR_INVALID_ARG;
    *out = nullptr;
    auto* n = new ccs_mpnn_s();
    n->ctx = c;
    bool ok = cudaMalloc(&n->master, kParams * 4) == cudaSuccess && cudaMalloc(&n->w16, kParams * 2) == cudaSuccess &&
              cudaMalloc(&n->grad, kParams * 4) == cudaSuccess && cudaMalloc(&n->m, kParams * 4) == cudaSuccess &&
              cudaMalloc(&n->v, kParams * 4) == cudaSuccess;
    if (!ok) {
      ccs_mpnn_free(n);
      return CCS_ERR_OOM;
    }
    // He-style uniform init from a 64-bit LCG; biases zero
    std::vector<float> h(kParams, 0.f);
    uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto uni = [&]() {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      return (float)((st >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
    };
    auto fill = [&](int off, int rows, int cols) {
      const float a = std::sqrt(6.f / (float)cols);
      for (int i = 0; i < rows * cols; ++i) h[off + i] = a * uni();
    };
    fill(oWin, kH, kIn);
    for (int l = 0; l < kLayers; ++l) {
      fill(oLayer + l * kLayerSize, kH, kH);
      fill(oLayer + l * kLayerSize + kH * kH, kH, kH);
    }
    fill(oWr1, kH, kR);
    fill(oWr2, 1, kH);
    if (ccs_mpnn_set_params(c, n, h.data()) != CCS_OK) {
      ccs_mpnn_free(n);
      return CCS_ERR_CUDA;
    }
    cudaMemset(n->m, 0, kParams * 4);
    cudaMemset(n->v, 0, kParams * 4);
    *out = n;
    return CCS_OK;
  });
}

void ccs_mpnn_free(ccs_mpnn n) {
  if (!n) return;
  cudaFree(n->master);
  cudaFree(n->w16);
  cudaFree(n->grad);
  cudaFree(n->m);
  cudaFree(n->v);
  delete n;
}

int ccs_mpnn_params(ccs_ctx c, ccs_mpnn n, float* out) {
  return abi_guard([](int code, const char*) { return code; }, [&]() -> int {
    if (!c || !n || !out) return CCS_ERR_INVALID_ARG;
    cudaStreamSynchronize(c_stream(c));
    return cudaMemcpy(out, n->master, kParams * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? CCS_OK : CCS_ERR_CUDA;
  });
}

int ccs_mpnn_set_params(ccs_ctx c, ccs_mpnn n, const float* in) {
  return abi_guard([](int code, const char*) { return code; }, [&]() -> int {
    if (!c || !n || !in) return CCS_ERR_INVALID_ARG;
    if (cudaMemcpy(n->master, in, kParams * 4, cudaMemcpyHostToDevice) != cudaSuccess) return CCS_ERR_CUDA;
    to_half<<<blocks(kParams), 256>>>(n->master, n->w16, kParams); note_launch();
    n->step = 0;
    return cudaDeviceSynchronize() == cudaSuccess ? CCS_OK : CCS_ERR_CUDA;
  });
}

int ccs_mpnn_forward(ccs_ctx c, ccs_mpnn n, const ccs_graph_batch* b, float* pred) {
  return abi_guard([](int code, const char*) { return code; }, [&]() -> int {
    if (!c || !n || !b || !pred || b->n_graphs <= 0) return CCS_ERR_INVALID_ARG;
    cudaStream_t s = c_stream(c);
    Batch d;
    int rc = upload_batch(b, nullptr, s, d);
    if (rc != CCS_OK) return rc;
    forward(n, d, s);
    if (cudaMemcpyAsync(pred, d.y, d.g * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CCS_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? CCS_OK : CCS_ERR_CUDA;
  });
}

int ccs_mpnn_gradient(ccs_ctx c, ccs_mpnn n, const ccs_graph_batch* b, const float* target, float* loss,
                      float* grad) {
  return abi_guard([](int code, const char*) { return code; }, [&]() -> int {
    if (!c || !n || !b || !target || b->n_graphs <= 0) return CCS_ERR_INVALID_ARG;
    cudaStream_t s = c_stream(c);
    Batch d;
    int rc = upload_batch(b, target, s, d);
    if (rc != CCS_OK) return rc;
    forward(n, d, s);
    backward(n, d, s);
    if (loss && cudaMemcpyAsync(loss, d.loss, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CCS_ERR_CUDA;
    if (grad && cudaMemcpyAsync(grad, n->grad, kParams * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return CCS_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? CCS_OK : CCS_ERR_CUDA;
  });
}

int ccs_mpnn_train_step(ccs_ctx c, ccs_mpnn n, const ccs_graph_batch* b, const float* target, float lr,
                        float* loss) {
  return abi_guard([](int code, const char*) { return code; }, [&]() -> int {
    if (!c || !n || !b || !target || b->n_graphs <= 0) return CCS_ERR_INVALID_ARG;
    cudaStream_t s = c_stream(c);
    Batch d;
    int rc = upload_batch(b, target, s, d);
    if (rc != CCS_OK) return rc;
    forward(n, d, s);
    backward(n, d, s);
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
    adam<<<blocks(kParams), 256, 0, s>>>(n->master, n->w16, n->grad, n->m, n->v, kParams, lr, b1, b2, c1, c2, 1e-8f); note_launch();
    if (loss && cudaMemcpyAsync(loss, d.loss, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CCS_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? CCS_OK : CCS_ERR_CUDA;
  });
}

}  // extern "C"

namespace ccs {
// Predict log times for a batch (used by the learned cut choice).
int mpnn_predict(ccs_mpnn n, const ccs_graph_batch* b, float* pred) { return ccs_mpnn_forward(n->ctx, n, b, pred); }
}  // namespace ccs
