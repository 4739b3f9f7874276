// Non-Clifford fragments (K4): complex64 statevectors of 2^n amplitudes in
// shared memory (the paper hands these fragments to an exact statevector
// simulator, Sec. V-B).  A variant is (preparations, the fragment's gates U,
// output basis changes), so an item (one preparation combination and a
// range of basis combinations) runs U once and then, for each basis
// combination, applies the output basis changes to a copy of the state.  Gates arrive fused into 2x2 / 4x4 unitaries; each
// gate reads one buffer and writes the other (ping-pong), one output
// amplitude per thread and pass, one barrier per gate.  Outputs per
// variant: the exact marginal on A_f and the Z-string values, both reduced
// in a fixed order (deterministic).
#include "kernels.cuh"

namespace ccs {

namespace {

__device__ __forceinline__ unsigned insert_zero(unsigned t, int pos) {
  return ((t >> pos) << (pos + 1)) | (t & ((1u << pos) - 1u));
}

__device__ __forceinline__ float2 cmul(float re, float im, float2 a) {
  return make_float2(re * a.x - im * a.y, re * a.y + im * a.x);
}

// One-qubit op on wire a: M row-major, M[r][c] at m[2 (2 r + c)].
__device__ __forceinline__ void apply_1q(const float2* __restrict__ src, float2* __restrict__ dst, unsigned N, int a,
                                         const float* m) {
  for (unsigned i = threadIdx.x; i < N; i += blockDim.x) {
    const unsigned r = (i >> a) & 1u, i0 = i & ~(1u << a);
    const float* row = m + 4 * r;
    const float2 x0 = src[i0], x1 = src[i0 | (1u << a)];
    const float2 p = cmul(row[0], row[1], x0), q = cmul(row[2], row[3], x1);
    dst[i] = make_float2(p.x + q.x, p.y + q.y);
  }
}

// Two-qubit op on wires (a, b): local index c = bit_a + 2 bit_b, M[r][c] at
// m[2 (4 r + c)].
__device__ __forceinline__ void apply_2q(const float2* __restrict__ src, float2* __restrict__ dst, unsigned N, int a,
                                         int b, const float* m) {
  const unsigned ma = 1u << a, mb = 1u << b;
  for (unsigned i = threadIdx.x; i < N; i += blockDim.x) {
    const unsigned r = ((i >> a) & 1u) | (((i >> b) & 1u) << 1), i00 = i & ~(ma | mb);
    const float* row = m + 8 * r;
    const float2 x0 = src[i00], x1 = src[i00 | ma], x2 = src[i00 | mb], x3 = src[i00 | ma | mb];
    const float2 p0 = cmul(row[0], row[1], x0), p1 = cmul(row[2], row[3], x1);
    const float2 p2 = cmul(row[4], row[5], x2), p3 = cmul(row[6], row[7], x3);
    dst[i] = make_float2((p0.x + p1.x) + (p2.x + p3.x), (p0.y + p1.y) + (p2.y + p3.y));
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

__global__ void __launch_bounds__(512) statevector_kernel(DevPlan P, DevRes R, int max_n) {
  extern __shared__ float2 sv_smem[];
  float2* buf[3] = {sv_smem, sv_smem + (1u << max_n), sv_smem + (2u << max_n)};
  NCOp* ops_s = reinterpret_cast<NCOp*>(sv_smem + (3u << max_n));
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
    const int n = F.n, qin = F.qin, qout = F.qout, nA = F.nA, nz = F.nz;
    const int n_prep = 1 << (2 * qin), n_basis = F.nv / n_prep;
    const int pc = it.y % n_prep, b0 = it.y / n_prep, b1 = min(n_basis, b0 + P.nc_basis_chunk);
    const unsigned N = 1u << n;
    const int op0 = P.moments[F.mom_off], op1 = P.moments[F.mom_off + F.n_moments];
    int cur = 0;
    for (unsigned i = tid; i < N; i += blockDim.x) buf[0][i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
    __syncthreads();
    for (int o = 0; o < qin; ++o) {
      apply_1q(buf[cur], buf[cur ^ 1], N, P.wires[F.qin_off + o], P.prep_mats + 8 * digit_in(pc, o));
      cur ^= 1;
      __syncthreads();
    }
    for (int c0 = op0; c0 < op1; c0 += kOpStage) {
      const int cnt = min(kOpStage, op1 - c0);
      const int* src = reinterpret_cast<const int*>(P.nops + F.ops_off + c0);
      int* dst = reinterpret_cast<int*>(ops_s);
      for (int i = tid; i < cnt * (int)(sizeof(NCOp) / 4); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      for (int o = 0; o < cnt; ++o) {
        const NCOp& op = ops_s[o];
        if (op.b < 0) apply_1q(buf[cur], buf[cur ^ 1], N, op.a, op.m);
        else apply_2q(buf[cur], buf[cur ^ 1], N, op.a, op.b, op.m);
        cur ^= 1;
        __syncthreads();
      }
    }
    // U |prep> stays in buf[cur]; each basis combination works in the other two
    const float2* psiU = buf[cur];
    float2* w0 = buf[cur ^ 1];
    float2* w1 = buf[3 - cur - (cur ^ 1)];
    for (int j = tid; j < nA; j += blockDim.x) s_abit[j] = 1u << P.wires[F.A_off + j];
    for (int o = tid; o < qout; o += blockDim.x) s_qm[o] = 1u << P.wires[F.qout_off + o];
    __syncthreads();
    unsigned amask = 0;
    for (int j = 0; j < nA; ++j) amask |= s_abit[j];
    const unsigned rest = (N - 1) & ~amask;
    const unsigned ncomp = 1u << (n - nA);
    for (int bc = b0; bc < b1; ++bc) {
      const int v = pc + n_prep * bc;
      const float2* psi = psiU;
      float2* wa = w0;
      float2* wb = w1;
      for (int o = 0; o < qout; ++o) {
        apply_1q(psi, wa, N, P.wires[F.qout_off + o], P.basis_mats + 8 * digit_out(v, qin, o));
        __syncthreads();
        psi = wa;
        float2* t = wa; wa = wb; wb = t;
      }
      // probabilities into a free buffer (not psiU, not psi)
      float* pr = reinterpret_cast<float*>(psi == w0 ? w1 : w0);
      for (unsigned i = tid; i < N; i += blockDim.x) pr[i] = psi[i].x * psi[i].x + psi[i].y * psi[i].y;
      __syncthreads();
      // marginal on A: one warp per output, lanes over its completions, then a
      // fixed shuffle tree
      float* d = R.dist + F.dist_off + ((long long)v << nA);
      for (unsigned y = warp; y < (1u << nA); y += nwarps) {
        unsigned base = 0;
        for (int j = 0; j < nA; ++j)
          if ((y >> j) & 1u) base |= s_abit[j];
        float acc = 0.f;
        for (unsigned c = lane; c < ncomp; c += 32) {
          unsigned idx = base, cc = c;          // deposit c's bits into the positions of `rest`
          for (unsigned rm = rest; rm && cc; rm &= rm - 1, cc >>= 1)
            if (cc & 1u) idx |= rm & (0u - rm);
          acc += pr[idx];
        }
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) d[y] = acc;
      }
      // Z-string values <Z_S> = sum_x (-1)^{|x & S|} p(x): the Walsh-Hadamard
      // transform of the probabilities, in place
      if (nz > 0) {
        __syncthreads();
        for (int h = 0; h < n; ++h) {
          for (unsigned t = tid; t < (N >> 1); t += blockDim.x) {
            const unsigned i0 = insert_zero(t, h), i1 = i0 | (1u << h);
            const float x0 = pr[i0], x1 = pr[i1];
            pr[i0] = x0 + x1;
            pr[i1] = x0 - x1;
          }
          __syncthreads();
        }
        for (int z0 = 0; z0 < nz; z0 += kZChunk) {
          const int zc = min(kZChunk, nz - z0);
          for (int k = tid; k < zc; k += blockDim.x) {
            unsigned zm = 0;
            for (int q = P.zoffs[F.zw_off + z0 + k]; q < P.zoffs[F.zw_off + z0 + k + 1]; ++q) zm ^= 1u << P.wires[q];
            s_zm[k] = zm;
          }
          __syncthreads();
          for (int ev = tid; ev < (zc << qout); ev += blockDim.x) {
            const int k = ev >> qout, u = ev & ((1 << qout) - 1);
            unsigned zm = s_zm[k];
            for (int o = 0; o < qout; ++o)
              if ((u >> o) & 1) zm ^= s_qm[o];
            R.zval[F.zval_off + ((long long)v * nz + z0 + k) * (1 << qout) + u] = pr[zm];
          }
          __syncthreads();
        }
      }
      __syncthreads();
    }
  }
}

cudaError_t launch_statevector(const DevPlan& p, const DevRes& r, int max_n, int threads, int grid,
                               cudaStream_t s) {
  if (p.n_items_nc == 0) return cudaSuccess;

  const size_t smem = ((size_t)24 << max_n) + (size_t)kOpStage * sizeof(NCOp);
  cudaError_t err = cudaFuncSetAttribute(statevector_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  statevector_kernel<<<grid, threads, smem, s>>>(p, r, max_n); note_launch();
  return cudaGetLastError();
}

}  // namespace ccs
