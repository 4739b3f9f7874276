// Non-Clifford fragments (K4): one complex64 statevector of 2^n amplitudes per
// variant in shared memory (the paper hands these fragments to an exact
// statevector simulator, Sec. V-B).  Gates arrive fused into 2x2 / 4x4
// unitaries; each is applied by all threads, one amplitude pair or quad per
// thread, with a barrier between ops.  Outputs: the exact marginal on A_f and
// the Z-string values, both reduced in a fixed order (deterministic).
#include "kernels.cuh"

namespace ccs {

namespace {

__device__ __forceinline__ unsigned insert_zero(unsigned t, int pos) {
  return ((t >> pos) << (pos + 1)) | (t & ((1u << pos) - 1u));
}

__device__ __forceinline__ float2 cmul(float re, float im, float2 a) {
  return make_float2(re * a.x - im * a.y, re * a.y + im * a.x);
}

__device__ void apply_1q(float2* psi, int n, int a, const float* m) {
  const unsigned half = 1u << (n - 1);
  for (unsigned t = threadIdx.x; t < half; t += blockDim.x) {
    const unsigned i0 = insert_zero(t, a), i1 = i0 | (1u << a);
    const float2 a0 = psi[i0], a1 = psi[i1];
    const float2 p = cmul(m[0], m[1], a0), q = cmul(m[2], m[3], a1);
    const float2 r = cmul(m[4], m[5], a0), s = cmul(m[6], m[7], a1);
    psi[i0] = make_float2(p.x + q.x, p.y + q.y);
    psi[i1] = make_float2(r.x + s.x, r.y + s.y);
  }
}

__device__ void apply_2q(float2* psi, int n, int a, int b, const float* m) {
  const unsigned quarter = 1u << (n - 2);
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  for (unsigned t = threadIdx.x; t < quarter; t += blockDim.x) {
    const unsigned i00 = insert_zero(insert_zero(t, lo), hi);
    unsigned idx[4] = {i00, i00 | (1u << a), i00 | (1u << b), i00 | (1u << a) | (1u << b)};
    float2 in[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) in[k] = psi[idx[k]];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float2 t2 = cmul(m[2 * (r * 4 + c)], m[2 * (r * 4 + c) + 1], in[c]);
        acc.x += t2.x;
        acc.y += t2.y;
      }
      psi[idx[r]] = acc;
    }
  }
}

__device__ __forceinline__ int digit_in(int v, int i) {
  for (int t = 0; t < i; ++t) v /= 4;
  return v % 4;
}
__device__ __forceinline__ int digit_out(int v, int qin, int i) {
  for (int t = 0; t < qin; ++t) v /= 4;
  for (int t = 0; t < i; ++t) v /= 3;
  return v % 3;
}

}  // namespace

constexpr int kOpStage = 128;   // fused ops staged in shared memory at a time
constexpr int kZChunk = 256;    // Z-string masks built per pass

__global__ void __launch_bounds__(256) statevector_kernel(DevPlan P, DevRes R, int max_n) {
  extern __shared__ float2 psi[];
  NCOp* ops_s = reinterpret_cast<NCOp*>(psi + (1u << max_n));
  __shared__ int s_item;
  __shared__ unsigned s_abit[kMaxMeas];     // bit of each A wire in the amplitude index
  __shared__ unsigned s_zm[kZChunk];        // Z masks of a chunk of Z-strings
  __shared__ unsigned s_qm[kMaxCuts];       // bit of each quantum output
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(&R.work[1], 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= P.n_items_nc) break;
    const int2 it = P.items_nc[item];
    const FragDev& F = P.frags[it.x];
    const int v = it.y, n = F.n;
    const unsigned N = 1u << n;
    for (unsigned i = tid; i < N; i += blockDim.x) psi[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
    __syncthreads();
    for (int o = 0; o < F.qin; ++o) {
      apply_1q(psi, n, P.wires[F.qin_off + o], P.prep_mats + 8 * digit_in(v, o));
      __syncthreads();
    }
    const int op0 = P.moments[F.mom_off], op1 = P.moments[F.mom_off + F.n_moments];
    for (int c0 = op0; c0 < op1; c0 += kOpStage) {
      const int cnt = min(kOpStage, op1 - c0);
      const int* src = reinterpret_cast<const int*>(P.nops + F.ops_off + c0);
      int* dst = reinterpret_cast<int*>(ops_s);
      for (int i = tid; i < cnt * (int)(sizeof(NCOp) / 4); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      for (int o = 0; o < cnt; ++o) {
        const NCOp& op = ops_s[o];
        if (op.b < 0) apply_1q(psi, n, op.a, op.m);
        else apply_2q(psi, n, op.a, op.b, op.m);
        __syncthreads();
      }
    }
    for (int o = 0; o < F.qout; ++o) {
      apply_1q(psi, n, P.wires[F.qout_off + o], P.basis_mats + 8 * digit_out(v, F.qin, o));
      __syncthreads();
    }
    // marginal on A: each output sums its completions in index order
    const int nA = F.nA;
    for (int j = tid; j < nA; j += blockDim.x) s_abit[j] = 1u << P.wires[F.A_off + j];
    for (int o = tid; o < F.qout; o += blockDim.x) s_qm[o] = 1u << P.wires[F.qout_off + o];
    __syncthreads();
    unsigned amask = 0;
    for (int j = 0; j < nA; ++j) amask |= s_abit[j];
    float* d = R.dist + F.dist_off + ((long long)v << nA);
    for (unsigned y = tid; y < (1u << nA); y += blockDim.x) {
      unsigned base = 0;
      for (int j = 0; j < nA; ++j)
        if ((y >> j) & 1u) base |= s_abit[j];
      float acc = 0.f;
      const unsigned rest = (N - 1) & ~amask;
      for (unsigned c = 0;; c = (c - rest) & rest) {     // subsets of `rest`, ascending
        const float2 a = psi[base | c];
        acc += a.x * a.x + a.y * a.y;
        if (c == rest) break;
      }
      d[y] = acc;
    }
    // Z-string values <Z_S> = sum_x (-1)^{|x & S|} p(x): the Walsh-Hadamard
    // transform of the probabilities, in place over the amplitude buffer
    if (F.nz > 0) {
      // psi -> p into the low half of the same buffer: block-wide rounds (a
      // uniform barrier count); round b writes floats [b, b + blockDim), i.e.
      // amplitudes below b + blockDim, all read before the round's barrier
      float* pr = reinterpret_cast<float*>(psi);
      for (unsigned b0 = 0; b0 < N; b0 += blockDim.x) {
        const unsigned i = b0 + tid;
        float pv = 0.f;
        if (i < N) {
          const float2 a = psi[i];
          pv = a.x * a.x + a.y * a.y;
        }
        __syncthreads();
        if (i < N) pr[i] = pv;
        __syncthreads();
      }
      for (int h = 0; h < n; ++h) {
        for (unsigned t = tid; t < (N >> 1); t += blockDim.x) {
          const unsigned i0 = insert_zero(t, h), i1 = i0 | (1u << h);
          const float x0 = pr[i0], x1 = pr[i1];
          pr[i0] = x0 + x1;
          pr[i1] = x0 - x1;
        }
        __syncthreads();
      }
      for (int z0 = 0; z0 < F.nz; z0 += kZChunk) {
        const int zc = min(kZChunk, F.nz - z0);
        for (int k = tid; k < zc; k += blockDim.x) {
          unsigned zm = 0;
          for (int q = P.zoffs[F.zw_off + z0 + k]; q < P.zoffs[F.zw_off + z0 + k + 1]; ++q) zm ^= 1u << P.wires[q];
          s_zm[k] = zm;
        }
        __syncthreads();
        for (int ev = tid; ev < (zc << F.qout); ev += blockDim.x) {
          const int k = ev >> F.qout, u = ev & ((1 << F.qout) - 1);
          unsigned zm = s_zm[k];
          for (int o = 0; o < F.qout; ++o)
            if ((u >> o) & 1) zm ^= s_qm[o];
          R.zval[F.zval_off + ((long long)v * F.nz + z0 + k) * (1 << F.qout) + u] = pr[zm];
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_statevector(const DevPlan& p, const DevRes& r, int max_n, int threads, int grid,
                               cudaStream_t s) {
  if (p.n_items_nc == 0) return cudaSuccess;

  const size_t smem = ((size_t)8 << max_n) + (size_t)kOpStage * sizeof(NCOp);
  cudaError_t err = cudaFuncSetAttribute(statevector_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  statevector_kernel<<<grid, threads, smem, s>>>(p, r, max_n); note_launch();
  return cudaGetLastError();
}

}  // namespace ccs
