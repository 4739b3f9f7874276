// Fold of variant data into fragment tensors (K5) and the contraction over the
// 4^k cut index (K6 / K7), Sec. III-B and V-C.
//
// On a cut wire rho = 1/2 sum_P Tr(P rho) P.  Upstream, Tr(P .) is read in
// basis beta(P) (Z for I and Z) with outcome weight lambda_P(b) = 1 for I and
// (-1)^b otherwise; downstream, P is expanded in prepared states with weights
// mu(P, s): I = (1, 1, 0, 0), X = (-1, -1, 2, 0), Y = (-1, -1, 0, 2),
// Z = (1, -1, 0, 0) over (|0>, |1>, |+>, |+i>).  Hence
//   T_f(o, P) = sum_s prod_i mu(P_in_i, s_i) sum_b prod_j lambda(P_out_j, b_j) p_(s,beta)(o, b)
//   p(o)      = 2^-k sum_P prod_f T_f(o_f, P|f).
#include "kernels.cuh"

#include <cuda_bf16.h>

namespace ccs {

namespace {

__device__ __forceinline__ int find_seg(const long long* prefix, int nseg, long long g) {
  int lo = 0, hi = nseg;          // prefix[lo] <= g < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Decode fragment-local Pauli index P into per-input / per-output Paulis.
struct PauliSplit {
  int pin[kMaxCuts], pout[kMaxCuts];
};

__device__ __forceinline__ void split_P(const FragDev& F, int P, PauliSplit& s) {
  for (int j = 0; j < F.n_slots; ++j) {
    const int pj = (P >> (2 * j)) & 3, code = F.slot_code[j];
    if ((code >> 8) == 0) s.pin[code & 255] = pj;
    else s.pout[code & 255] = pj;
  }
}

// Walk the preparation tuples with nonzero weight for the inputs' Paulis.
// Returns the number of tuples; fills vin[] and coef[] lazily via callback.
template <class Fn>
__device__ __forceinline__ void for_each_prep(const FragDev& F, const PauliSplit& ps, Fn fn) {
  // options per input: I/Z -> {|0>, |1>}, X -> {|+>, |0>, |1>}, Y -> {|+i>, |0>, |1>}
  int cnt[kMaxCuts], total = 1;
  for (int i = 0; i < F.qin; ++i) {
    cnt[i] = (ps.pin[i] == 1 || ps.pin[i] == 2) ? 3 : 2;
    total *= cnt[i];
  }
  for (int t = 0; t < total; ++t) {
    int rem = t, vin = 0, mul = 1;
    double coef = 1.0;
    for (int i = 0; i < F.qin; ++i) {
      const int c = rem % cnt[i];
      rem /= cnt[i];
      const int P = ps.pin[i];
      int s;
      double w;
      if (P == 0) { s = c; w = 1.0; }
      else if (P == 3) { s = c; w = c ? -1.0 : 1.0; }
      else { s = c == 0 ? (P == 1 ? 2 : 3) : c - 1; w = c == 0 ? 2.0 : -1.0; }
      vin += s * mul;
      mul *= 4;
      coef *= w;
    }
    fn(vin, coef);
  }
}

__device__ __forceinline__ float to_bf16f(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
// sum += p with the low part the rounding loses kept in comp (Neumaier)
__device__ __forceinline__ void neumaier(float& sum, float& comp, float p) {
  const float t = sum + p;                     // keep the low part the sum loses
  comp += fabsf(sum) >= fabsf(p) ? (sum - t) + p : (p - t) + sum;
  sum = t;
}

}  // namespace

__global__ void fold_kernel(DevPlan P, DevRes R, EvalParams E, const int* fidx, const long long* prefix,
                            int nf, long long total) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int fs = find_seg(prefix, nf, g);
    const FragDev& F = P.frags[fidx[fs]];
    const long long loc = g - prefix[fs];
    const int S2 = 2 * F.n_slots;
    const int o = (int)(loc >> S2), Pi = (int)(loc & ((1ll << S2) - 1));
    PauliSplit ps;
    split_P(F, Pi, ps);
    int vout = 0, mul = 1;
    for (int j = 0; j < F.qout; ++j) {
      const int beta = ps.pout[j] == 1 ? 0 : ps.pout[j] == 2 ? 1 : 2;   // I,Z->Z(2) X->0 Y->1
      vout += beta * mul;
      mul *= 3;
    }
    int vstride = 1;
    for (int i = 0; i < F.qin; ++i) vstride *= 4;
    const bool use_counts = F.clifford && E.mode == CCS_SAMPLED;
    const int m = F.m, nA = F.nA;
    double acc = 0.0;
    for_each_prep(F, ps, [&](int vin, double coef) {
      const long long v = vin + (long long)vstride * vout;
      for (int b = 0; b < (1 << F.qout); ++b) {
        int neg = 0;
        for (int j = 0; j < F.qout; ++j) neg ^= (ps.pout[j] != 0) & ((b >> j) & 1);
        const long long y = ((long long)v << nA) | ((long long)b << m) | o;
        const double val = use_counts ? (double)R.counts[F.counts_off + y] * E.inv_shots
                                      : (double)R.dist[F.dist_off + y];
        acc += neg ? -coef * val : coef * val;
      }
    });
    R.T[F.T_off + loc] = (float)acc;
  }
}

// Contraction operands.  Writing the hub's tensor through its preparations,
//   T_h(o, P) = sum_s prod_{input cuts i} mu(P_i, s_i) Q_h(o, s, P_out),
//   Q_h(o, s, P_out) = sum_b prod_j lambda(P_out_j, b_j) p_(s, beta(P_out))(o, b),
// moves the mu weights onto the fragment upstream of each hub input cut:
//   p(o) = 2^-k sum_{s, P_out} Q_h(o, s, P_out) prod_l T'_l,
//   T'_l(o_l, ...) = sum over P at the cuts where l feeds the hub of
//                    prod mu(P_i, s_i) T_l(o_l, P).
// Q_h reads one variant per entry (no sum over preparations) and T'_l is
// small, so the large hub tensor is never formed.
__global__ void qfold_kernel(DevPlan P, DevRes R, EvalParams E, const int* fidx, const long long* prefix, int nf,
                             long long total) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int fs = find_seg(prefix, nf, g);
    const FragDev& F = P.frags[fidx[fs]];
    const long long loc = g - prefix[fs];     // hub operand stored transposed: loc = D * 2^m + o
    const int o = (int)(loc & ((1ll << F.m) - 1)), D = (int)(loc >> F.m);
    int pout[kMaxCuts];
    long long vin = 0;
    for (int j = 0; j < F.n_slots; ++j) {
      const int d = (D >> (2 * j)) & 3, code = F.slot_code[j], idx = code & 255;
      if ((code >> 8) == 0) vin += (long long)d << (2 * idx);
      else pout[idx] = d;
    }
    long long vout = 0, mul = 1;
    for (int j = 0; j < F.qout; ++j) {
      vout += (pout[j] == 1 ? 0 : pout[j] == 2 ? 1 : 2) * mul;
      mul *= 3;
    }
    const long long v = vin + (vout << (2 * F.qin));
    const bool use_counts = F.clifford && E.mode == CCS_SAMPLED;
    double acc = 0.0;
    for (int b = 0; b < (1 << F.qout); ++b) {
      int neg = 0;
      for (int j = 0; j < F.qout; ++j) neg ^= (pout[j] != 0) & ((b >> j) & 1);
      const long long y = (v << F.nA) | ((long long)b << F.m) | o;
      const double val = use_counts ? (double)R.counts[F.counts_off + y] * E.inv_shots : (double)R.dist[F.dist_off + y];
      acc += neg ? -val : val;
    }
    R.TQ[F.T_off + loc] = (float)acc;
  }
}

__global__ void prime_kernel(DevPlan P, DevRes R, const int* fidx, const long long* prefix, int nf,
                             long long total) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int fs = find_seg(prefix, nf, g);
    const FragDev& F = P.frags[fidx[fs]];
    const long long loc = g - prefix[fs];
    const int S2 = 2 * F.n_slots;
    const long long row = (loc >> S2) << S2;
    const int D = (int)(loc & ((1ll << S2) - 1));
    // slots where this fragment feeds the hub (its quantum outputs) carry a
    // preparation digit s; expand each into the Paulis with mu(P, s) != 0
    int outs[kMaxCuts], nout = 0, base = D;
    for (int j = 0; j < F.n_slots; ++j)
      if ((F.slot_code[j] >> 8) == 1) {
        outs[nout++] = j;
        base &= ~(3 << (2 * j));
      }
    int total_c = 1;
    int cnt[kMaxCuts];
    for (int t = 0; t < nout; ++t) {
      const int sdig = (D >> (2 * outs[t])) & 3;
      cnt[t] = sdig < 2 ? 4 : 1;
      total_c *= cnt[t];
    }
    double acc = 0.0;
    for (int c = 0; c < total_c; ++c) {
      int rem = c, Pidx = base;
      double coef = 1.0;
      for (int t = 0; t < nout; ++t) {
        const int sdig = (D >> (2 * outs[t])) & 3;
        int pj;
        double w;
        if (sdig < 2) {
          pj = rem % 4;
          rem /= 4;
          w = (pj == 0) ? 1.0 : (pj == 3) ? (sdig == 0 ? 1.0 : -1.0) : -1.0;   // I, X, Y, Z
        } else {
          pj = sdig == 2 ? 1 : 2;    // |+> -> X, |+i> -> Y, weight 2
          w = 2.0;
        }
        Pidx |= pj << (2 * outs[t]);
        coef *= w;
      }
      acc += coef * (double)R.T[F.T_off + row + Pidx];
    }
    R.TQ[F.T_off + loc] = (float)acc;
  }
}

cudaError_t launch_operands(const DevPlan& p, const DevRes& r, const EvalParams& e, const FoldSet& hubs,
                            const FoldSet& others, cudaStream_t s) {
  if (hubs.total > 0) {
    const long long blocks = (hubs.total + 255) / 256;
    qfold_kernel<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, s>>>(p, r, e, hubs.fidx,
                                                                                 hubs.t_prefix, hubs.nf,
                                                                                 hubs.total); note_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (others.total > 0) {
    const long long blocks = (others.total + 255) / 256;
    prime_kernel<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, s>>>(p, r, others.fidx,
                                                                                 others.t_prefix, others.nf,
                                                                                 others.total); note_launch();
  }
  return cudaGetLastError();
}

// --- contraction over the 4^k cut index ------------------------------------
// For a star (hub h + leaves), p(o) = 2^-k sum_P T_h[o_h, P] R[P, o_l] with
// R[P, o_l] = prod_leaves T_l[o_l|l, P|l] (leaf outputs concatenated in
// fragment order; cut-free fragments contribute their P-independent factor).
// Stars that contract_kernel does not take leaf by leaf (the tensor-core path
// and stars too wide for a slice) go through the GEMM chain: R is built once
// (it is the GEMM's B operand), then a tiled GEMM with split-K writes FP32
// partial tiles, and the partials are summed in FP64 in a fixed order, scaled
// by 2^-k and scattered to marginal order.  BF16 mode rounds both operands to
// bf16 (as a bf16 tensor-core GEMM would) with FP32 accumulation.

// Whether a problem's FP32 contraction takes the first-leaf streaming path
// (dense rows, full cut-index range; its Rrest table then replaces R).
static __host__ __device__ bool fact_path(const ProblemDev& Pb, int precision, int stitched, bool full_range) {
  return Pb.stream && Pb.fact && !Pb.direct && precision == CCS_FP32 && !stitched && full_range;
}

__global__ void build_r_kernel(DevPlan P, DevRes R, int precision, const long long* prefix, int np,
                               long long total, float* scratch, uint16_t* rt_scratch, int stitched, int full_range) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int pi = find_seg(prefix, np, g);
    const ProblemDev& Pb = P.problems[pi];
    const long long loc = g - prefix[pi];
    const long long Pp = loc / Pb.N;
    const long long ol = loc - Pp * Pb.N;
    // a streamed stitched hub reads no R row of a zero operand row; a problem
    // on the first-leaf path builds its own smaller table instead of R
    if (stitched && Pb.stream && Pb.hub_qrow_off >= 0 && !R.qnz[Pb.hub_qrow_off + Pp]) continue;
    if (fact_path(Pb, precision, stitched, full_range != 0) && !(rt_scratch && Pb.tc)) continue;
    float v = 1.f;
    int off = 0;
    for (int l = 0; l < Pb.n_frags; ++l) {
      if (l == Pb.hub) continue;
      const FragDev& L = P.frags[Pb.frag0 + l];
      const int x = (int)((ol >> off) & ((1ll << L.m) - 1));
      off += L.m;
      int pl = 0;
      for (int i = 0; i < L.n_slots; ++i) pl |= (int)((Pp >> (2 * L.slot_cut[i])) & 3) << (2 * i);
      v *= R.TQ[L.T_off + ((long long)x << (2 * L.n_slots)) + pl];
    }
    if (precision == CCS_BF16) v = to_bf16f(v);
    scratch[Pb.r_off + loc] = v;
    if (precision == CCS_BF16 && Pb.tc && rt_scratch)   // R'^T for the tensor-core GEMM
      reinterpret_cast<__nv_bfloat16*>(rt_scratch)[Pb.rt_off + ol * Pb.K + Pp] = __float2bfloat16_rn(v);
  }
}

constexpr int kTK = 16;

// Split-K GEMM tile: TM x TN outputs (multiples of 4), one 4x4 register
// micro-tile per thread, A staged k-major and B row-major in shared memory so
// each k step is two float4 reads and 16 FMAs.
__global__ void __launch_bounds__(256) gemm_splitk_kernel(DevPlan P, DevRes R, int precision,
                                                          const long long* blk_prefix, int np,
                                                          long long total_blocks, float* scratch, int skip_tc,
                                                          KRange kr) {
  extern __shared__ __align__(16) float sm[];
  for (long long b = blockIdx.x; b < total_blocks; b += gridDim.x) {
    const int pi = find_seg(blk_prefix, np, b);
    const ProblemDev& Pb = P.problems[pi];
    if ((skip_tc && Pb.tc) || Pb.stream) continue;   // done by the tensor-core or the streaming GEMM
    const FragDev& Hb = P.frags[Pb.frag0 + Pb.hub];
    long long loc = b - blk_prefix[pi];
    const int nt = (int)(loc % Pb.ntiles); loc /= Pb.ntiles;
    const int mt = (int)(loc % Pb.mtiles); loc /= Pb.mtiles;
    const int split = (int)loc;
    const int TM = Pb.TM, TN = Pb.TN, M = Pb.M, N = Pb.N;
    const long long K = Pb.K;
    const long long kchunk = (K + Pb.splits - 1) / Pb.splits;
    const long long s0 = split * kchunk;     // this split's terms within the requested range
    const long long k0 = max(s0, kr.lo_of(K)), k1 = min(min(s0 + kchunk, K), kr.hi_of(K));
    float* As = sm;                  // kTK x TM
    float* Bs = sm + kTK * TM;       // kTK x TN
    const HubView At = hub_view(R, Hb, Hb.T_off);   // the hub's Q stored transposed: K x M, row-major
    const float* Bm = scratch + Pb.r_off;    // K x N, row-major
    const int tn4 = TN >> 2;
    const bool act = (int)threadIdx.x < (TM >> 2) * tn4;
    const int mi = act ? ((int)threadIdx.x / tn4) * 4 : 0, ni = act ? ((int)threadIdx.x % tn4) * 4 : 0;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (long long kk = k0; kk < k1; kk += kTK) {
      for (int t = threadIdx.x; t < TM * kTK; t += blockDim.x) {
        const int m = t % TM, k = t / TM;
        const long long gm = (long long)mt * TM + m, gk = kk + k;
        float v = (gm < M && gk < k1) ? At.at(gk * M + gm) : 0.f;
        if (precision == CCS_BF16) v = to_bf16f(v);
        As[k * TM + m] = v;
      }
      for (int t = threadIdx.x; t < kTK * TN; t += blockDim.x) {
        const int k = t / TN, n = t % TN;
        const long long gn = (long long)nt * TN + n, gk = kk + k;
        Bs[k * TN + n] = (gn < N && gk < k1) ? Bm[gk * N + gn] : 0.f;
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int k = 0; k < kTK; ++k) {
          const float4 av = *reinterpret_cast<const float4*>(As + k * TM + mi);
          const float4 bv = *reinterpret_cast<const float4*>(Bs + k * TN + ni);
          const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a4[i], b4[j], acc[i][j]);
        }
      }
      __syncthreads();
    }
    if (act) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const long long gm = (long long)mt * TM + mi + i, gn = (long long)nt * TN + ni + j;
          if (gm < M && gn < N) scratch[Pb.part_off + ((long long)split * M + gm) * N + gn] = acc[i][j];
        }
    }
  }
}

// Streaming CUDA-core GEMM of a wide hub operand: the partial
//   C[m][n] = sum_{k in one K range} Q^T[k][m] R[k][n]
// of one split.  Thread t of CTA (mb, split) owns the hub outputs
// m = 4 (mb blockDim + t) .. +3 and every column n: one 16-byte streaming
// load of Q^T per row (a CTA reads blockDim x 16 contiguous bytes of each
// row, each byte once), the R rows of the range staged in shared memory and
// read as broadcasts, eight rows of loads in flight.  FP32 FMA per split;
// the splits are summed in FP64 by reduce_scatter_kernel.  BF16 mode rounds
// the hub values to bf16 (R is rounded when it is built).
constexpr int kStreamChunk = 256;   // R rows staged per pass

// Four consecutive hub operand entries as floats: FP32 as stored, or the
// int16 count sums themselves (the streaming GEMMs apply 1/shots once to
// each accumulator at the end: exact when the shots are a power of two).
__device__ __forceinline__ float4 hub4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 hub4(const int16_t* p) {
  const short4 v = *reinterpret_cast<const short4*>(p);
  return make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
}
// VW consecutive operand entries as one load (16/8/4-byte FP32, 8/4/2-byte
// int16), kept packed until used; the caller guarantees the alignment.
template <class T, int VW> struct RawVec;
template <> struct RawVec<float, 4> { using type = float4; };
template <> struct RawVec<float, 2> { using type = float2; };
template <> struct RawVec<float, 1> { using type = float; };
template <> struct RawVec<int16_t, 4> { using type = int2; };
template <> struct RawVec<int16_t, 2> { using type = int; };
template <> struct RawVec<int16_t, 1> { using type = short; };
__device__ __forceinline__ float raw_at(const float4& q, int v, float) {
  return v == 0 ? q.x : v == 1 ? q.y : v == 2 ? q.z : q.w;
}
__device__ __forceinline__ float raw_at(const float2& q, int v, float) { return v == 0 ? q.x : q.y; }
__device__ __forceinline__ float raw_at(float q, int, float) { return q; }
__device__ __forceinline__ float raw_at(int q, int v, float sc) {
  return (float)(v ? (q >> 16) : (int)(short)(q & 0xffff)) * sc;
}
__device__ __forceinline__ float raw_at(const int2& q, int v, float sc) { return raw_at(v < 2 ? q.x : q.y, v & 1, sc); }
__device__ __forceinline__ float raw_at(short q, int, float sc) { return (float)q * sc; }
__device__ __forceinline__ float4 hub4_stream(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 hub4_stream(const int16_t* p) {
  const int2 w = __ldcs(reinterpret_cast<const int2*>(p));
  return make_float4((float)(short)(w.x & 0xffff), (float)(short)((unsigned)w.x >> 16), (float)(short)(w.y & 0xffff),
                     (float)(short)((unsigned)w.y >> 16));
}

template <int NN>
__device__ __forceinline__ void stream_fma(float (&acc)[4][NN], float4 a, const float* rrow, int bf16) {
  if (bf16) { a.x = to_bf16f(a.x); a.y = to_bf16f(a.y); a.z = to_bf16f(a.z); a.w = to_bf16f(a.w); }
  float rv[NN];
  if constexpr (NN >= 4) {
#pragma unroll
    for (int j = 0; j < NN; j += 4) {
      const float4 r4 = *reinterpret_cast<const float4*>(rrow + j);
      rv[j] = r4.x; rv[j + 1] = r4.y; rv[j + 2] = r4.z; rv[j + 3] = r4.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < NN; ++j) rv[j] = rrow[j];
  }
#pragma unroll
  for (int j = 0; j < NN; ++j) {
    acc[0][j] = fmaf(a.x, rv[j], acc[0][j]);
    acc[1][j] = fmaf(a.y, rv[j], acc[1][j]);
    acc[2][j] = fmaf(a.z, rv[j], acc[2][j]);
    acc[3][j] = fmaf(a.w, rv[j], acc[3][j]);
  }
}

template <int NN, class T>
__global__ void __launch_bounds__(256, 2) gemm_stream_kernel(const T* __restrict__ At, float sc,
                                                             const float* __restrict__ Rm, int M, long long K,
                                                             long long kchunk, int mblocks, float* __restrict__ part,
                                                             int bf16, const uint8_t* __restrict__ live, KRange kr) {
  __shared__ __align__(16) float Rs[kStreamChunk * NN];
  __shared__ __align__(8) uint8_t Ls[kStreamChunk];     // row flags of the chunk (stitched operands)
  const int mb = blockIdx.x % mblocks, split = blockIdx.x / mblocks;
  const long long s0 = (long long)split * kchunk;     // this split's rows within the requested range
  const long long k0 = max(s0, kr.lo_of(K)), k1 = min(min(K, s0 + kchunk), kr.hi_of(K));
  const int m = 4 * (mb * (int)blockDim.x + (int)threadIdx.x);
  const bool act = m < M;
  float acc[4][NN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NN; ++j) acc[i][j] = 0.f;
  for (long long kc = k0; kc < k1; kc += kStreamChunk) {
    const int rows = (int)min((long long)kStreamChunk, k1 - kc);
    __syncthreads();                       // the previous chunk's rows are consumed
    if (live)
      for (int i = threadIdx.x; i < kStreamChunk; i += blockDim.x) Ls[i] = i < rows ? live[kc + i] : 0;
    for (int i = threadIdx.x; i < rows * NN; i += blockDim.x)
      if (!live || live[kc + i / NN]) Rs[i] = Rm[kc * NN + i];
    __syncthreads();
    if (!act) continue;
    const T* ap = At + kc * M + m;
    int r = 0;
    for (; r + 8 <= rows; r += 8) {
      if (live) {        // rows flagged zero are skipped (they may never have been written)
        const unsigned long long l8 = *reinterpret_cast<const unsigned long long*>(Ls + r);
        if (!l8) continue;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if ((l8 >> (8 * u)) & 0xffull)
            stream_fma<NN>(acc, hub4_stream(ap + (long long)(r + u) * M), Rs + (r + u) * NN, bf16);
        continue;
      }
      float4 a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = hub4_stream(ap + (long long)(r + u) * M);
#pragma unroll
      for (int u = 0; u < 8; ++u) stream_fma<NN>(acc, a[u], Rs + (r + u) * NN, bf16);
    }
    for (; r < rows; ++r)
      if (!live || Ls[r])
        stream_fma<NN>(acc, hub4_stream(ap + (long long)r * M), Rs + r * NN, bf16);
  }
  if (!act) return;
  float* dst = part + ((long long)split * M + m) * NN;    // 4 x NN contiguous floats
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NN; ++j) dst[i * NN + j] = acc[i][j] * sc;
}

// The same split-K product for dense operands with the loads moved off the
// threads: one producer lane streams the CTA's slice of each Q^T row
// (blockDim' x 16 bytes, contiguous) and the R rows of a stage into a
// shared-memory ring with cp.async.bulk (the TMA engine), completing on the
// stage's mbarrier; the consumer warps wait for a stage, take their float4
// of each row from shared memory (conflict-free) and release the stage.
// Every wait is bounded by a clock budget: on expiry the kernel sets status
// bit 8, stops issuing, waits (bounded) for its copies in flight and writes
// zero partials.
constexpr int kBulkRows = 8, kBulkStages = 3;
constexpr unsigned long long kBulkWaitBudget = 2000000000ull;   // ~1 s of SM clocks

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bulk_wait(uint64_t* bar, uint32_t phase) {
  const unsigned long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kBulkWaitBudget) return false;
  }
}

template <int NN, class T>
__global__ void __launch_bounds__(288, 2) gemm_stream_bulk_kernel(const T* __restrict__ At, float sc,
                                                                 const float* __restrict__ Rm, int M, long long K,
                                                                 long long kchunk, int mblocks, float* __restrict__ part,
                                                                 int bf16, KRange kr, unsigned* status) {
  extern __shared__ __align__(128) uint8_t bulk_smem[];
  const int nc = (int)blockDim.x - 32;                  // consumer threads, 4 hub outputs each
  const int row_bytes = nc * 4 * (int)sizeof(T);
  T* A_s = reinterpret_cast<T*>(bulk_smem);                                           // [stage][row][4 nc]
  float* R_s = reinterpret_cast<float*>(bulk_smem + kBulkStages * kBulkRows * row_bytes);   // [stage][row][NN]
  uint64_t* full = reinterpret_cast<uint64_t*>(bulk_smem + kBulkStages * kBulkRows * (row_bytes + NN * 4));
  uint64_t* empty = full + kBulkStages;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kBulkStages);
  const int mb = blockIdx.x % mblocks, split = blockIdx.x / mblocks;
  const long long s0 = (long long)split * kchunk;
  const long long k0 = max(s0, kr.lo_of(K)), k1 = min(min(K, s0 + kchunk), kr.hi_of(K));
  const long long nrows = k1 > k0 ? k1 - k0 : 0;
  const int nstage = (int)((nrows + kBulkRows - 1) / kBulkRows);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, cw = nc >> 5;
  const int m0 = mb * nc * 4;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kBulkStages; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(cw) : "memory");
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == cw) {                                     // producer warp
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nstage; ++i) {
        const int st = i % kBulkStages;
        if (i >= kBulkStages && !bulk_wait(&empty[st], ((i / kBulkStages) - 1) & 1)) {
          atomicOr(status, 8u);
          *abort_flag = 1;
        }
        if (*abort_flag) break;
        const long long r0 = k0 + (long long)i * kBulkRows;
        const int rows = (int)min((long long)kBulkRows, k1 - r0);
        const uint32_t bytes = (uint32_t)(rows * row_bytes + rows * NN * 4);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[st])), "r"(bytes)
                     : "memory");
        for (int r = 0; r < rows; ++r)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(A_s + ((size_t)st * kBulkRows + r) * nc * 4)),
              "l"(At + (r0 + r) * M + m0), "r"(row_bytes), "r"(smem_u32(&full[st]))
              : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(R_s + (size_t)st * kBulkRows * NN)),
            "l"(Rm + r0 * NN), "r"((uint32_t)(rows * NN * 4)), "r"(smem_u32(&full[st]))
            : "memory");
        issued = i + 1;
      }
      if (*abort_flag)      // let copies already issued land before the shared memory is released
        for (int i = max(0, issued - kBulkStages); i < issued; ++i) bulk_wait(&full[i % kBulkStages], (i / kBulkStages) & 1);
    }
    return;
  }
  float acc[4][NN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NN; ++j) acc[i][j] = 0.f;
  for (int i = 0; i < nstage; ++i) {
    const int st = i % kBulkStages;
    bool ok = !*abort_flag && bulk_wait(&full[st], (i / kBulkStages) & 1);
    ok = __all_sync(0xffffffffu, ok) != 0;
    if (!ok) {
      if (lane == 0) { atomicOr(status, 8u); *abort_flag = 1; }
      break;
    }
    const long long r0 = k0 + (long long)i * kBulkRows;
    const int rows = (int)min((long long)kBulkRows, k1 - r0);
    const T* as = A_s + (size_t)st * kBulkRows * nc * 4 + threadIdx.x * 4;
    const float* rs = R_s + (size_t)st * kBulkRows * NN;
    for (int r = 0; r < rows; ++r) stream_fma<NN>(acc, hub4(as + (size_t)r * nc * 4), rs + r * NN, bf16);
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[st])) : "memory");
  }
  const int m = m0 + 4 * (int)threadIdx.x;
  if (m >= M) return;
  const bool good = !*abort_flag;
  float* dst = part + ((long long)split * M + m) * NN;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NN; ++j) dst[i * NN + j] = good ? acc[i][j] * sc : 0.f;
}

// --- the first leaf contracted while streaming --------------------------
// For a star whose first leaf l1 (the lowest leaf-output bits) owns s1 <= 2
// cuts and N1 <= 2 marginal outputs, the Kronecker operand factorises as
//   R[P][x1 + N1 xr] = T'_l1[x1][g1(P)] Rrest[rest(P)][xr],
// g1 the leaf's cut digits of P and rest the others.  So the G1 = 4^s1 rows
// of one rest value (a group) contract first against the leaf's table,
//   Y[m][x1] = sum_g1 Q^T[P(g1, rest)][m] T'_l1[x1][g1],
// and only then meet the other leaves: acc[m][x1 + N1 xr] += Y[m][x1]
// Rrest[rest][xr] -- 4 (N1 G1 + N) FMA per group and 4 hub outputs instead
// of 4 G1 N: 12 instead of 64 per operand row at config 3.  Rows are fetched
// one group per pipeline stage by the TMA engine (bulk copies of each row's
// CTA slice), as in gemm_stream_bulk_kernel; FP32, dense rows, full range.
constexpr int kFactRrStage = 4096;   // floats of Rrest rows a CTA stages in shared memory

struct FactDigits {
  int ndig1, ndigr;
  int dig1[kMaxCuts], digr[kMaxCuts];
};

__device__ __forceinline__ long long scatter_digits(long long v, int nd, const int* pos) {
  long long p = 0;
  for (int j = 0; j < nd; ++j) p |= ((v >> (2 * j)) & 3ll) << (2 * pos[j]);
  return p;
}

// Rrest[group][xr] = prod over the leaves after l1 of T'_l[x_l][g_l(P)], P the
// group's rest digits (the first leaf's digits zero), x_l the leaves' bits of xr.
__global__ void build_rrest_kernel(DevPlan P, DevRes R, ProblemDev Pb, FactDigits dg, float* __restrict__ rr,
                                   long long total) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long grp = g / Pb.NR;
    const int xr = (int)(g - grp * Pb.NR);
    const long long Pp = scatter_digits(grp, dg.ndigr, dg.digr);
    float v = 1.f;
    int off = 0;
    for (int l = 0; l < Pb.n_frags; ++l) {
      if (l == Pb.hub || l == Pb.fl1) continue;
      const FragDev& L = P.frags[Pb.frag0 + l];
      const int x = (xr >> off) & ((1 << L.m) - 1);
      off += L.m;
      int pl = 0;
      for (int i = 0; i < L.n_slots; ++i) pl |= (int)((Pp >> (2 * L.slot_cut[i])) & 3) << (2 * i);
      v *= R.TQ[L.T_off + ((long long)x << (2 * L.n_slots)) + pl];
    }
    rr[g] = v;
  }
}

template <int N1, int NR, class T>
__global__ void __launch_bounds__(288, 2) gemm_fact_bulk_kernel(const T* __restrict__ At, float sc,
                                                                const float* __restrict__ T1, int G1,
                                                                const float* __restrict__ Rr, int M, long long ngroups,
                                                                long long gchunk, int mblocks, int stages,
                                                                float* __restrict__ part, FactDigits dg,
                                                                unsigned* status) {
  constexpr int N = N1 * NR;
  extern __shared__ __align__(128) uint8_t fact_smem[];
  const int nc = (int)blockDim.x - 32;                  // consumer threads, 4 hub outputs each
  const int row_bytes = nc * 4 * (int)sizeof(T);
  const int stage_bytes = G1 * row_bytes;
  T* A_s = reinterpret_cast<T*>(fact_smem);
  float* T1s = reinterpret_cast<float*>(fact_smem + (size_t)stages * stage_bytes);   // [x1][g1]
  uint64_t* full = reinterpret_cast<uint64_t*>(T1s + ((N1 * G1 + 1) & ~1));
  uint64_t* empty = full + stages;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + stages);
  long long* pg = reinterpret_cast<long long*>(empty + stages + 1);   // [G1]: the leaf digits' row offsets
  int* digr = reinterpret_cast<int*>(pg + G1);                         // the other digits' cut positions
  float* Rrs = reinterpret_cast<float*>(digr + kMaxCuts);              // this CTA's Rrest rows, when staged
  const int mb = blockIdx.x % mblocks, split = blockIdx.x / mblocks;
  const long long gr0 = (long long)split * gchunk, gr1 = min(ngroups, gr0 + gchunk);
  const int nstage = gr1 > gr0 ? (int)(gr1 - gr0) : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, cw = nc >> 5;
  const int m0 = mb * nc * 4;
  for (int i = threadIdx.x; i < N1 * G1; i += blockDim.x) T1s[i] = T1[i];
  for (int g = threadIdx.x; g < G1; g += blockDim.x) pg[g] = scatter_digits(g, dg.ndig1, dg.dig1);
  const bool rr_staged = gchunk * NR <= kFactRrStage;
  if (rr_staged)
    for (long long i = threadIdx.x; i < (long long)nstage * NR; i += blockDim.x) Rrs[i] = Rr[gr0 * NR + i];
  if (threadIdx.x < dg.ndigr) digr[threadIdx.x] = dg.digr[threadIdx.x];
  if (threadIdx.x == 0) {
    for (int i = 0; i < stages; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(1) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(cw) : "memory");
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == cw) {                                     // producer warp: lanes < G1 copy one row each
    int issued = 0;
    for (int i = 0; i < nstage; ++i) {
      const int st = i % stages;
      bool ok = true;
      if (lane == 0 && i >= stages && !bulk_wait(&empty[st], ((i / stages) - 1) & 1)) {
        atomicOr(status, 8u);
        *abort_flag = 1;
      }
      ok = __shfl_sync(0xffffffffu, (int)!*abort_flag, 0) != 0;
      if (!ok) break;
      if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[st])),
                     "r"((uint32_t)stage_bytes)
                     : "memory");
      __syncwarp();
      long long prest = 0;
      const long long grp = gr0 + i;
      for (int j = 0; j < dg.ndigr; ++j) prest |= ((grp >> (2 * j)) & 3ll) << (2 * digr[j]);
      for (int g = lane; g < G1; g += 32)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(A_s + ((size_t)st * G1 + g) * nc * 4)),
            "l"(At + (prest | pg[g]) * M + m0), "r"(row_bytes), "r"(smem_u32(&full[st]))
            : "memory");
      issued = i + 1;
    }
    if (lane == 0 && *abort_flag)      // let copies already issued land before the shared memory is released
      for (int i = max(0, issued - stages); i < issued; ++i) bulk_wait(&full[i % stages], (i / stages) & 1);
    return;
  }
  float acc[4][N];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) acc[i][j] = 0.f;
  for (int i = 0; i < nstage; ++i) {
    const int st = i % stages;
    bool ok = !*abort_flag && bulk_wait(&full[st], (i / stages) & 1);
    ok = __all_sync(0xffffffffu, ok) != 0;
    if (!ok) {
      if (lane == 0) { atomicOr(status, 8u); *abort_flag = 1; }
      break;
    }
    float y[4][N1];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int x = 0; x < N1; ++x) y[a][x] = 0.f;
    const T* as = A_s + (size_t)st * G1 * nc * 4 + threadIdx.x * 4;
    using Raw = typename RawVec<T, 4>::type;
    for (int g = 0; g < G1; g += 4) {          // G1 = 4^s1: four rows' loads in flight, kept packed
      Raw v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const Raw*>(as + (size_t)(g + u) * nc * 4);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int x = 0; x < N1; ++x) {
          const float t = T1s[x * G1 + g + u];
#pragma unroll
          for (int a = 0; a < 4; ++a) y[a][x] = fmaf(raw_at(v[u], a, 1.f), t, y[a][x]);
        }
    }
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[st])) : "memory");
    float rv[NR];
    if (rr_staged) {
#pragma unroll
      for (int xr = 0; xr < NR; ++xr) rv[xr] = Rrs[(long long)i * NR + xr];
    } else {
#pragma unroll
      for (int xr = 0; xr < NR; ++xr) rv[xr] = __ldg(Rr + (gr0 + i) * NR + xr);
    }
#pragma unroll
    for (int xr = 0; xr < NR; ++xr)
#pragma unroll
      for (int x = 0; x < N1; ++x)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][x + N1 * xr] = fmaf(y[a][x], rv[xr], acc[a][x + N1 * xr]);
  }
  const int m = m0 + 4 * (int)threadIdx.x;
  if (m >= M) return;
  const bool good = !*abort_flag;
  float* dst = part + ((long long)split * M + m) * N;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) dst[i * N + j] = good ? acc[i][j] * sc : 0.f;
}

template <int N1, int NR, class T>
static cudaError_t launch_fact_t(const T* At, float sc, const DevPlan& p, const DevRes& r, const ProblemDev& Pb,
                                 float* scratch, cudaStream_t s) {
  FactDigits dg{};
  dg.ndig1 = Pb.ndig1;
  dg.ndigr = Pb.ndigr;
  for (int i = 0; i < kMaxCuts; ++i) { dg.dig1[i] = Pb.dig1[i]; dg.digr[i] = Pb.digr[i]; }
  const long long ngroups = Pb.K / Pb.G1;
  float* rr = scratch + Pb.r_off;                 // the group table takes R's place
  build_rrest_kernel<<<(unsigned)std::min<long long>((ngroups * Pb.NR + 255) / 256, 65535), 256, 0, s>>>(
      p, r, Pb, dg, rr, ngroups * Pb.NR);
  note_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const long long gchunk = (ngroups + Pb.ssplits - 1) / Pb.ssplits;
  const long long splits = Pb.ssplits;            // every split writes its partial (zero when empty)
  const int stage_bytes = Pb.G1 * Pb.sthreads * 4 * (int)sizeof(T);
  const int stages = std::max(2, std::min(4, (112 << 10) / stage_bytes));
  const size_t rr_floats = gchunk * Pb.NR <= kFactRrStage ? (size_t)gchunk * Pb.NR : 0;
  const size_t smem = (size_t)stages * stage_bytes + (size_t)((N1 * Pb.G1 + 1) & ~1) * 4 + 2 * stages * 8 + 8 +
                      (size_t)Pb.G1 * 8 + kMaxCuts * 4 + rr_floats * 4 + 16;
  err = cudaFuncSetAttribute(gemm_fact_bulk_kernel<N1, NR, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  gemm_fact_bulk_kernel<N1, NR, T><<<(unsigned)(Pb.smblocks * splits), Pb.sthreads + 32, smem, s>>>(
      At, sc, r.TQ + Pb.fl1_T_off, Pb.G1, rr, Pb.M, ngroups, gchunk, Pb.smblocks, stages, scratch + Pb.part_off, dg,
      r.status);
  note_launch();
  return cudaGetLastError();
}

template <int NN, class T>
static cudaError_t launch_stream_nn(const T* At, float sc, const float* Rm, const ProblemDev& Pb, float* part,
                                    int bf16, const uint8_t* live, KRange kr, unsigned* status, cudaStream_t s) {
  const long long kchunk = (Pb.K + Pb.ssplits - 1) / Pb.ssplits;
  const long long splits = Pb.ssplits;         // every split writes its partial (zero when its range is empty)
  const bool bulk = NN >= 4 && live == nullptr && Pb.sthreads % 32 == 0 && status != nullptr &&
                    (reinterpret_cast<uintptr_t>(At) & 15) == 0 && (reinterpret_cast<uintptr_t>(Rm) & 15) == 0 &&
                    (Pb.M * sizeof(T)) % 16 == 0;
  if (bulk) {   // dense operand: rows streamed by the TMA engine into a shared-memory ring
    const size_t smem =
        (size_t)kBulkStages * kBulkRows * (Pb.sthreads * 4 * sizeof(T) + NN * 4) + 2 * kBulkStages * 8 + 16;
    cudaError_t err =
        cudaFuncSetAttribute(gemm_stream_bulk_kernel<NN, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    gemm_stream_bulk_kernel<NN, T><<<(unsigned)(Pb.smblocks * splits), Pb.sthreads + 32, smem, s>>>(
        At, sc, Rm, Pb.M, Pb.K, kchunk, Pb.smblocks, part, bf16, kr, status);
  } else {
    gemm_stream_kernel<NN, T><<<(unsigned)(Pb.smblocks * splits), Pb.sthreads, 0, s>>>(
        At, sc, Rm, Pb.M, Pb.K, kchunk, Pb.smblocks, part, bf16, live, kr);
  }
  note_launch();
  return cudaGetLastError();
}

// The hub operand of a problem as the host sees it (a Clifford hub's sampled
// operand holds int16 count sums).
static HubView hub_host_view(const DevRes& r, const ProblemDev& Pb) {
  HubView v;
  v.f = r.TQ + Pb.hub_T_off;
  v.h = (r.hub_i16 && Pb.hub_qrow_off >= 0) ? reinterpret_cast<const int16_t*>(r.TQ + Pb.hub_T_off) : nullptr;
  v.scale = r.hub_scale;
  return v;
}

template <class T>
static cudaError_t launch_stream_t(const T* At, float sc, const DevRes& r, const ProblemDev& Pb, float* scratch,
                                   int bf16, int stitched, KRange kr, cudaStream_t s) {
  const float* Rm = scratch + Pb.r_off;
  float* part = scratch + Pb.part_off;
  const uint8_t* live = (stitched && Pb.hub_qrow_off >= 0) ? r.qnz + Pb.hub_qrow_off : nullptr;
  switch (Pb.N) {
    case 1: return launch_stream_nn<1>(At, sc, Rm, Pb, part, bf16, live, kr, r.status, s);
    case 2: return launch_stream_nn<2>(At, sc, Rm, Pb, part, bf16, live, kr, r.status, s);
    case 4: return launch_stream_nn<4>(At, sc, Rm, Pb, part, bf16, live, kr, r.status, s);
    case 8: return launch_stream_nn<8>(At, sc, Rm, Pb, part, bf16, live, kr, r.status, s);
    case 16: return launch_stream_nn<16>(At, sc, Rm, Pb, part, bf16, live, kr, r.status, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class T>
static cudaError_t launch_fact_any(const T* At, float sc, const DevPlan& p, const DevRes& r, const ProblemDev& Pb,
                                   float* scratch, cudaStream_t s) {
  switch (Pb.N1 * 32 + Pb.NR) {
    case 32 + 1: return launch_fact_t<1, 1>(At, sc, p, r, Pb, scratch, s);
    case 32 + 2: return launch_fact_t<1, 2>(At, sc, p, r, Pb, scratch, s);
    case 32 + 4: return launch_fact_t<1, 4>(At, sc, p, r, Pb, scratch, s);
    case 32 + 8: return launch_fact_t<1, 8>(At, sc, p, r, Pb, scratch, s);
    case 32 + 16: return launch_fact_t<1, 16>(At, sc, p, r, Pb, scratch, s);
    case 64 + 1: return launch_fact_t<2, 1>(At, sc, p, r, Pb, scratch, s);
    case 64 + 2: return launch_fact_t<2, 2>(At, sc, p, r, Pb, scratch, s);
    case 64 + 4: return launch_fact_t<2, 4>(At, sc, p, r, Pb, scratch, s);
    case 64 + 8: return launch_fact_t<2, 8>(At, sc, p, r, Pb, scratch, s);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t launch_fact(const DevPlan& p, const DevRes& r, const ProblemDev& Pb, float* scratch,
                               cudaStream_t s) {
  const HubView v = hub_host_view(r, Pb);
  if (v.h) return launch_fact_any(v.h, v.scale, p, r, Pb, scratch, s);
  return launch_fact_any(v.f, 1.0f, p, r, Pb, scratch, s);
}

static cudaError_t launch_stream(const DevRes& r, const ProblemDev& Pb, float* scratch, int bf16, int stitched,
                                 KRange kr, cudaStream_t s) {
  const HubView v = hub_host_view(r, Pb);
  if (v.h) return launch_stream_t(v.h, v.scale, r, Pb, scratch, bf16, stitched, kr, s);
  return launch_stream_t(v.f, 1.0f, r, Pb, scratch, bf16, stitched, kr, s);
}

// BF16 K-major copy of a hub operand for the tensor-core GEMM:
// Qh[o][D] = bf16(Q^T[D][o]), through 64 x 64 shared-memory tiles: each
// warp reads 256 contiguous bytes of a Q^T row (o fastest) and writes 128
// contiguous bytes of a Qh row as bf16 pairs (D fastest).
__global__ void __launch_bounds__(256) hub_bf16_kernel(HubView QT, __nv_bfloat16* __restrict__ Qh, int M,
                                                       long long K) {
  __shared__ float tile[64][65];
  const long long tiles_d = (K + 63) / 64, tiles_o = (M + 63) / 64;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;   // 8 warps
  for (long long t = blockIdx.x; t < tiles_d * tiles_o; t += gridDim.x) {
    const long long d0 = (t / tiles_o) * 64;
    const int o0 = (int)(t % tiles_o) * 64;
    for (int r = warp; r < 64; r += 8) {            // rows of Q^T: 64 floats each, two per lane
      const long long d = d0 + r;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int o = o0 + lane + 32 * h;
        tile[r][lane + 32 * h] = (d < K && o < M) ? QT.at(d * M + o) : 0.f;
      }
    }
    __syncthreads();
    for (int r = warp; r < 64; r += 8) {            // rows of Qh: 64 bf16 each, one pair per lane
      const int o = o0 + r;
      const long long d = d0 + 2 * lane;
      if (o < M && d + 1 < K) {
        *reinterpret_cast<__nv_bfloat162*>(Qh + (long long)o * K + d) =
            __floats2bfloat162_rn(tile[2 * lane][r], tile[2 * lane + 1][r]);
      } else if (o < M && d < K) {
        Qh[(long long)o * K + d] = __float2bfloat16_rn(tile[2 * lane][r]);
      }
    }
    __syncthreads();
  }
}

// The split-K partials summed and scattered to marginal order.  A CTA takes
// 32 consecutive outputs (one per lane, so every load of a warp is one
// contiguous row segment); its 8 warps sum splits w, w + 8, ... with
// compensated FP32 sums (FP64 arithmetic is scarce on this GPU), and the
// warps' (sum, compensation) pairs are added in FP64 in warp order: a fixed
// order, many loads in flight.
__global__ void __launch_bounds__(256) reduce_scatter_kernel(DevPlan P, const long long* prefix, int np,
                                                             long long total, const float* scratch, double* marg_out,
                                                             int use_tc) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (long long base = blockIdx.x * 32ll; base < total; base += gridDim.x * 32ll) {
    const long long g = base + lane;
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
    int pi = -1;
    if (g < total) {
      pi = find_seg(prefix, np, g);
      const ProblemDev& Pb = P.problems[pi];
      if (Pb.direct || Pb.general) pi = -1;   // written by the leaf-by-leaf or the general contraction
      else {
        const long long loc = g - prefix[pi];
        const int splits = (Pb.stream && !(use_tc && Pb.tc)) ? Pb.ssplits : Pb.splits;
        const float* pp = scratch + Pb.part_off + loc;    // partial [split][m][n]: loc = m N + n
        const long long st = (long long)Pb.M * Pb.N;
        int s = w;
        for (; s + 24 < splits; s += 32) {    // four loads in flight
          const float v0 = pp[(long long)s * st], v1 = pp[(long long)(s + 8) * st];
          const float v2 = pp[(long long)(s + 16) * st], v3 = pp[(long long)(s + 24) * st];
          neumaier(s0, c0, v0);
          neumaier(s1, c1, v1);
          neumaier(s0, c0, v2);
          neumaier(s1, c1, v3);
        }
        for (; s < splits; s += 8) neumaier(s0, c0, pp[(long long)s * st]);
      }
    }
    red[w][lane] = ((double)s0 + (double)c0) + ((double)s1 + (double)c1);
    __syncthreads();
    if (w == 0 && pi >= 0) {
      const ProblemDev& Pb = P.problems[pi];
      double acc = red[0][lane];
#pragma unroll
      for (int j = 1; j < 8; ++j) acc += red[j][lane];
      const long long loc = g - prefix[pi];
      const long long m = loc / Pb.N, n = loc - m * Pb.N;
      long long o = 0;
      const FragDev& Hb = P.frags[Pb.frag0 + Pb.hub];
      for (int j = 0; j < Hb.m; ++j) o |= ((m >> j) & 1) << Hb.marg_pos[j];
      int off = 0;
      for (int l = 0; l < Pb.n_frags; ++l) {
        if (l == Pb.hub) continue;
        const FragDev& L = P.frags[Pb.frag0 + l];
        for (int j = 0; j < L.m; ++j) o |= ((n >> (off + j)) & 1) << L.marg_pos[j];
        off += L.m;
      }
      marg_out[Pb.marg_off + o] = ldexp(acc, -Pb.k);
    }
    __syncthreads();
  }
}

// Fragment descriptors of one problem, read once into shared memory so that
// the per-element loops below do no dependent global loads.
constexpr int kMaxProblemFrags = kMaxProblemFragments;   // checked when the plan is built
constexpr int kLeafStage = 2048;   // floats of a leaf table staged in shared memory
struct ProblemShared {
  int nf, hub, k;
  int m[kMaxProblemFrags], ns[kMaxProblemFrags];
  int slot_cut[kMaxProblemFrags][kMaxCuts];
  int marg_pos[kMaxProblemFrags][kMaxMarginal];
  long long T_off[kMaxProblemFrags];
};

__device__ void load_problem(const DevPlan& P, const ProblemDev& Pb, ProblemShared& S) {
  const int t = threadIdx.x;
  if (t == 0) { S.nf = Pb.n_frags; S.hub = Pb.hub; S.k = Pb.k; }
  if (t < Pb.n_frags) {
    const FragDev& L = P.frags[Pb.frag0 + t];
    S.m[t] = L.m;
    S.ns[t] = L.n_slots;
    S.T_off[t] = L.T_off;
    for (int i = 0; i < L.n_slots; ++i) S.slot_cut[t][i] = L.slot_cut[i];
    for (int j = 0; j < L.m; ++j) S.marg_pos[t][j] = L.marg_pos[j];
  }
}

// Slot digits of fragment l in cut index Pp.
__device__ __forceinline__ int frag_digits(const ProblemShared& S, int l, long long Pp) {
  int pl = 0;
  for (int i = 0; i < S.ns[l]; ++i) pl |= (int)((Pp >> (2 * S.slot_cut[l][i])) & 3) << (2 * i);
  return pl;
}

// T_f^S(zi, P) folded from the variants' Z-string values the way T_f is
// folded from their distributions: the preparation tuples of P's input
// Paulis (weights mu) at the output bases of P's output Paulis, each taking
// the value of Z_S times the observables of the outputs whose Pauli is not I.
__device__ float fold_z_value(const DevRes& R, const FragDev& F, int zi, int Pi) {
  PauliSplit ps;
  split_P(F, Pi, ps);
  int vout = 0, mul = 1, u = 0;
  for (int j = 0; j < F.qout; ++j) {
    const int beta = ps.pout[j] == 1 ? 0 : ps.pout[j] == 2 ? 1 : 2;
    vout += beta * mul;
    mul *= 3;
    if (ps.pout[j] != 0) u |= 1 << j;
  }
  int vstride = 1;
  for (int i = 0; i < F.qin; ++i) vstride *= 4;
  double acc = 0.0;
  for_each_prep(F, ps, [&](int vin, double coef) {
    const long long v = vin + (long long)vstride * vout;
    acc += coef * (double)R.zval[F.zval_off + (v * F.nz + zi) * (1 << F.qout) + u];
  });
  return (float)acc;
}

// <Z_S> = 2^-k sum_P prod_f T_f^S(P|f): one block per (problem, string),
// FP32 products, FP64 sums, fixed-order tree reduction; T_f^S is folded from
// the variants' Z values here (no separate fold pass).
__device__ __noinline__ void z_string_block(const DevPlan& P, const DevRes& R, const long long* prefix, int np, long long g,
                               ProblemShared& S, double* red, float* s_tz, int tz_cap, double* zexp_out, KRange kr) {
  const int pi = find_seg(prefix, np, g);
  const ProblemDev& Pb = P.problems[pi];
  const int zi = (int)(g - prefix[pi]);
  load_problem(P, Pb, S);
  __syncthreads();
  // every fragment's T_f^S(zi, .) folded once into shared memory when it fits
  int tz_tot = 0;
  for (int l = 0; l < S.nf; ++l) tz_tot += 1 << (2 * S.ns[l]);
  const bool staged = tz_tot <= tz_cap;
  if (staged) {
    for (int i = threadIdx.x; i < tz_tot; i += blockDim.x) {
      int l = 0, o = 0;
      while (i >= o + (1 << (2 * S.ns[l]))) { o += 1 << (2 * S.ns[l]); ++l; }
      s_tz[i] = fold_z_value(R, P.frags[Pb.frag0 + l], zi, i - o);
    }
    __syncthreads();
  }
  const long long K = 1ll << (2 * S.k);
  double part = 0.0;
  for (long long Pp = kr.lo_of(K) + threadIdx.x; Pp < kr.hi_of(K); Pp += blockDim.x) {
    float t = 1.f;
    int o = 0;
    for (int l = 0; l < S.nf; ++l) {
      const int pl = frag_digits(S, l, Pp);
      t *= staged ? s_tz[o + pl] : fold_z_value(R, P.frags[Pb.frag0 + l], zi, pl);
      o += 1 << (2 * S.ns[l]);
    }
    part += (double)t;
  }
  red[threadIdx.x] = part;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) zexp_out[Pb.zexp_off + zi] = ldexp(red[0], -S.k);
}

// Contraction of a star leaf by leaf (the tensor-network order of Sec.
// V-C), one CTA per slice of TM hub outputs (the contraction never mixes
// them), every intermediate in shared memory.
// Each cut belongs to exactly one leaf, so the cut index P splits into the
// leaves' digit groups g_l (a leaf's digits in its slot order, so g_l is
// the column index of T'_l).  Start from X[kc][m] = Q^T[P][m], kc the cut
// index with the groups in leaf order (the first leaf's group lowest); each
// leaf then replaces its group by its outputs:
//   Y[rest][outer + A x] = sum_g X[g + G rest][outer] T'_l[x][g],
// outer = (m, x_1, ..., x_{l-1}) of size A.  After the last leaf
// X[outer] = C[m][n], scaled by 2^-k and scattered to marginal order.
// 2^m K sum_l 2^(m_1+..+m_l) / 4^(s_1+..+s_l) multiply-adds instead of
// the 2^m K 2^(m_1+..+m_L) of the Kronecker GEMM.  Sums are compensated
// (Neumaier) FP32; operands are rounded to bf16 first in BF16 mode.
// Blocks after the problems compute the Z-string expectations.
// One operand entry as a float: FP32 as stored, or an int16 count sum times 1/shots.
__device__ __forceinline__ float hub_elem(const float* A, float, long long i) { return A[i]; }
__device__ __forceinline__ float hub_elem(const int16_t* A, float sc, long long i) { return (float)A[i] * sc; }

// The first leaf of a slice, read from the hub operand in global memory:
//   Y[r][x][m] = sum_g Q^T[kr(r) | kg(g)][m0 + m] T'[x][g]
// (r: the other leaves' digits, g: this leaf's, x: its outputs), each thread
// VW consecutive hub outputs (one vector load per row) and two outputs x
// (every operand load used twice), four rows in flight.
template <class T> constexpr int first_vec() { return sizeof(T) == 2 ? 4 : 2; }   // hub outputs per thread
constexpr int kFirstX = 2;      // leaf outputs per thread (1 or 2)
constexpr int kFirstRows = 4;   // operand rows in flight per thread (divides 4^slots)
template <int VW, int NX, class T, class Expand>
__device__ __forceinline__ void first_leaf_global(const T* __restrict__ At, float sc, int bf16, long long Mfull,
                                                  int lm, int lG, int ml, int lrest, long long klo, long long khi,
                                                  const float* tv, bool tv_rounded, const int* kg_tab,
                                                  const ProblemShared& S, int l, Expand expand, float* Y) {
  const int G = 1 << lG, lV = VW == 4 ? 2 : VW == 2 ? 1 : 0, lmv = lm - lV;
  const int nx = (NX == 2 && ml > 0) ? 2 : 1, lxc = nx == 2 ? ml - 1 : ml;
  const int lout = lm + ml;
  const int n_items = 1 << (lrest + lxc + lmv);
  for (int e = threadIdx.x; e < n_items; e += blockDim.x) {
    const int mv = e & ((1 << lmv) - 1);
    const int x0 = ((e >> lmv) & ((1 << lxc) - 1)) * nx;
    const int r = e >> (lmv + lxc);
    const int kr = expand(r << lG, l);
    float s0[VW], c0[VW], s1[NX == 2 ? VW : 1], c1[NX == 2 ? VW : 1];
#pragma unroll
    for (int v = 0; v < VW; ++v) { s0[v] = c0[v] = 0.f; if (NX == 2) s1[v] = c1[v] = 0.f; }
    const T* base = At + mv * VW;
    for (int g0 = 0; g0 < G; g0 += kFirstRows) {      // G = 4^slots >= 4 (a leaf without cuts is staged)
      using Raw = typename RawVec<T, VW>::type;
      Raw a[kFirstRows];
#pragma unroll
      for (int u = 0; u < kFirstRows; ++u) {
        const int g = g0 + u;
        int kg;
        if (kg_tab) kg = kg_tab[g];
        else {
          kg = 0;
          for (int i = 0; i < S.ns[l]; ++i) kg |= ((g >> (2 * i)) & 3) << (2 * S.slot_cut[l][i]);
        }
        const long long kk = (long long)(kr | kg);
        a[u] = (kk >= klo && kk < khi) ? __ldg(reinterpret_cast<const Raw*>(base + kk * Mfull)) : Raw{};
      }
#pragma unroll
      for (int u = 0; u < kFirstRows; ++u) {
        const int g = g0 + u;
        float t0 = tv[x0 * G + g], t1 = nx == 2 ? tv[(x0 + 1) * G + g] : 0.f;
        if (bf16 && !tv_rounded) { t0 = to_bf16f(t0); t1 = to_bf16f(t1); }
#pragma unroll
        for (int v = 0; v < VW; ++v) {
          float av = raw_at(a[u], v, sc);
          if (bf16) av = to_bf16f(av);
          neumaier(s0[v], c0[v], av * t0);
          if (NX == 2 && nx == 2) neumaier(s1[v], c1[v], av * t1);
        }
      }
    }
    float* y = Y + ((long long)r << lout) + mv * VW;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      y[((long long)x0 << lm) + v] = s0[v] + c0[v];
      if (NX == 2 && nx == 2) y[((long long)(x0 + 1) << lm) + v] = s1[v] + c1[v];
    }
  }
}

// One slice of TM hub outputs of one star, contracted leaf by leaf (the
// body of contract_kernel), for the hub operand's stored element type.
template <class T>
__device__ __forceinline__ void contract_item(const DevPlan& P, const DevRes& R, int precision, const ProblemDev& Pb,
                                              const T* __restrict__ At, float sc, int m0, int M, int lm, int Mfull,
                                              int K, long long klo, long long khi, ProblemShared& S, float* s_buf,
                                              int stage_floats, float* s_T, double* marg_out) {
  load_problem(P, Pb, S);
  __syncthreads();
  float* X = s_buf;
  float* Y = s_buf + stage_floats;
  // compact cut index (groups in leaf order, the first leaf's lowest) ->
  // cut index, for the digits of leaves from `from` on
  auto expand = [&](int kc, int from) -> int {
    int k = 0, rem = kc;
    for (int l = from; l < S.nf; ++l) {
      if (l == S.hub) continue;
      for (int i = 0; i < S.ns[l]; ++i) {
        k |= (rem & 3) << (2 * S.slot_cut[l][i]);
        rem >>= 2;
      }
    }
    return k;
  };
  int first = 0;
  while (first < S.nf && first == S.hub) ++first;
  // no leaf: the operand is the result; a first leaf without cuts: the operand
  // slice staged (it fits: every leaf's intermediate holds K x TM floats then)
  const bool staged0 = first >= S.nf || S.ns[first] == 0;
  if (staged0) {
    for (int t0 = threadIdx.x; t0 < K * M; t0 += 8 * blockDim.x) {   // 8 loads in flight per thread
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < K * M) {
          const long long kk = expand(t >> lm, 0);
          v[u] = (kk >= klo && kk < khi) ? hub_elem(At, sc, kk * Mfull + (t & (M - 1))) : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < K * M) X[t] = precision == CCS_BF16 ? to_bf16f(v[u]) : v[u];
      }
    }
  }
  int lA = lm, lrest = 2 * S.k;                // log2 of the outer and rest extents
  for (int l = first; l < S.nf; ++l) {
    if (l == S.hub) continue;
    const int lG = 2 * S.ns[l], G = 1 << lG, Nl = 1 << S.m[l];
    lrest -= lG;
    const bool tstaged = Nl * G <= kLeafStage;
    __syncthreads();                           // X complete; previous s_T consumed
    if (tstaged)
      for (int i = threadIdx.x; i < Nl * G; i += blockDim.x) {
        float v = R.TQ[S.T_off[l] + i];
        if (precision == CCS_BF16) v = to_bf16f(v);
        s_T[i] = v;
      }
    // the first leaf's digits in the cut index, tabulated behind its table when they fit
    int* kg_tab = nullptr;
    if (l == first && !staged0 && tstaged && Nl * G + G <= kLeafStage) {
      kg_tab = reinterpret_cast<int*>(s_T + Nl * G);
      for (int g = threadIdx.x; g < G; g += blockDim.x) {
        int kg = 0;
        for (int i = 0; i < S.ns[l]; ++i) kg |= ((g >> (2 * i)) & 3) << (2 * S.slot_cut[l][i]);
        kg_tab[g] = kg;
      }
    }
    __syncthreads();
    const int lout = lA + S.m[l], A = 1 << lA;
    if (l == first && !staged0) {
      const float* tv = tstaged ? s_T : R.TQ + S.T_off[l];
      if ((1 << lm) >= first_vec<T>())         // aligned vectors: T_off and m0 are multiples of TM
        first_leaf_global<first_vec<T>(), kFirstX>(At, sc, precision == CCS_BF16, Mfull, lm, lG, S.m[l], lrest, klo, khi, tv, tstaged,
                             kg_tab, S, l, expand, Y);
      else
        first_leaf_global<1, kFirstX>(At, sc, precision == CCS_BF16, Mfull, lm, lG, S.m[l], lrest, klo, khi, tv, tstaged,
                             kg_tab, S, l, expand, Y);
      float* tmp = X; X = Y; Y = tmp;
      lA = lout;
      continue;
    }
    for (int e = threadIdx.x; e < (1 << (lrest + lout)); e += blockDim.x) {
      const int r = e >> lout, rm = e & ((1 << lout) - 1);
      const int x = rm >> lA, outer = rm & (A - 1);
      float sum = 0.f, comp = 0.f;
      const float* xs = X + ((r << lG) << lA) + outer;
      const float* ts = tstaged ? s_T + x * G : nullptr;
      for (int g = 0; g < G; ++g) {
        float tv;
        if (tstaged) tv = ts[g];
        else {
          tv = R.TQ[S.T_off[l] + (long long)x * G + g];
          if (precision == CCS_BF16) tv = to_bf16f(tv);
        }
        neumaier(sum, comp, xs[g << lA] * tv);
      }
      Y[e] = sum + comp;
    }
    float* tmp = X; X = Y; Y = tmp;
    lA = lout;
  }
  // X[m + M n] = C[m][n]; marginal index = hub bits of m | leaf bits of n,
  // both tabulated in the free buffer (TM + N entries, within its size)
  const int hub = S.hub, N = 1 << (lA - lm);
  unsigned* orow = reinterpret_cast<unsigned*>(Y);
  unsigned* ocol = orow + M;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    unsigned o = 0;
    for (int j = 0; j < S.m[hub]; ++j) o |= ((unsigned)((m0 + m) >> j) & 1u) << S.marg_pos[hub][j];
    orow[m] = o;
  }
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    unsigned o = 0;
    int off = 0;
    for (int l = 0; l < S.nf; ++l) {
      if (l == hub) continue;
      for (int j = 0; j < S.m[l]; ++j) o |= ((unsigned)(n >> (off + j)) & 1u) << S.marg_pos[l][j];
      off += S.m[l];
    }
    ocol[n] = o;
  }
  __syncthreads();
  const double scale = ldexp(1.0, -S.k);       // exact: a power of two
  double* out = marg_out + Pb.marg_off;
  for (int t = threadIdx.x; t < (1 << lA); t += blockDim.x)
    out[orow[t & (M - 1)] | ocol[t >> lm]] = (double)X[t] * scale;
  __syncthreads();
}

__global__ void __launch_bounds__(512, 2) contract_kernel(DevPlan P, DevRes R, int precision,
                                                      const int2* direct_items, int n_direct, int stage_floats,
                                                      const long long* z_prefix, int np, long long z_total,
                                                      double* marg_out, double* zexp_out, KRange krg) {
  extern __shared__ __align__(16) float s_buf[];   // two buffers of stage_floats
  __shared__ double red[512];
  __shared__ ProblemShared S;
  __shared__ float s_T[kLeafStage];
  for (long long b = blockIdx.x; b < n_direct + z_total; b += gridDim.x) {
    if (b >= n_direct) {
      z_string_block(P, R, z_prefix, np, b - n_direct, S, red, s_T, kLeafStage, zexp_out, krg);
      __syncthreads();
      continue;
    }
    const int2 di = direct_items[b];
    const ProblemDev& Pb = P.problems[di.x];
    const int M = Pb.TM, lm = __ffs(M) - 1;      // this block's hub outputs; extents are powers of two
    const int m0 = di.y * M, Mfull = Pb.M;
    const int K = (int)Pb.K;
    const long long klo = krg.lo_of(K), khi = krg.hi_of(K);   // cut-index terms summed
    // the hub's Q stored transposed: K x Mfull, row-major (this slice's columns from m0),
    // FP32 or int16 count sums: one branch per slice, none per element
    const HubView hv = hub_view(R, P.frags[Pb.frag0 + Pb.hub], Pb.hub_T_off + m0);
    if (hv.h)
      contract_item(P, R, precision, Pb, hv.h, hv.scale, m0, M, lm, Mfull, K, klo, khi, S, s_buf, stage_floats, s_T,
                    marg_out);
    else
      contract_item(P, R, precision, Pb, hv.f, 1.0f, m0, M, lm, Mfull, K, klo, khi, S, s_buf, stage_floats, s_T,
                    marg_out);
  }
}

cudaError_t launch_fold(const DevPlan& p, const DevRes& r, const EvalParams& e, const FoldSet& f,
                        cudaStream_t s) {
  if (f.total == 0) return cudaSuccess;
  const long long blocks = (f.total + 255) / 256;
  fold_kernel<<<(unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8), 256, 0, s>>>(p, r, e, f.fidx, f.t_prefix, f.nf,
                                                                            f.total); note_launch();
  return cudaGetLastError();
}

// --- any topology ----------------------------------------------------------
// A problem with no fragment on every cut (a chain or a tree of fragments,
// Sec. V-C's general tensor network) is summed directly: for each output o,
//   p(o) = 2^-k sum_P prod_f T_f(o_f, P|f),
// one CTA per output, the cut index strided over its threads (FP32 products,
// compensated FP32 sums per thread, FP64 across threads in a fixed order).
// 4^k x 2^|o| x fragments reads: the general form, not a fast path.
__global__ void __launch_bounds__(256) general_contract_kernel(DevPlan P, DevRes R, int precision,
                                                               const long long* out_prefix, int np, long long total,
                                                               double* marg_out, KRange kr) {
  __shared__ double red[256];
  __shared__ ProblemShared S;
  for (long long b = blockIdx.x; b < total; b += gridDim.x) {
    const int pi = find_seg(out_prefix, np, b);
    const ProblemDev& Pb = P.problems[pi];
    if (!Pb.general) continue;                 // stars are contracted by the other kernels
    const long long o = b - out_prefix[pi];
    load_problem(P, Pb, S);
    __syncthreads();
    const long long K = Pb.K, lo = kr.lo_of(K), hi = kr.hi_of(K);
    float sum = 0.f, comp = 0.f;
    for (long long Pp = lo + threadIdx.x; Pp < hi; Pp += blockDim.x) {
      float t = 1.f;
      for (int l = 0; l < S.nf; ++l) {
        int of = 0;
        for (int j = 0; j < S.m[l]; ++j) of |= (int)((o >> S.marg_pos[l][j]) & 1) << j;
        float v = R.T[S.T_off[l] + ((long long)of << (2 * S.ns[l])) + frag_digits(S, l, Pp)];
        if (precision == CCS_BF16) v = to_bf16f(v);
        t *= v;
      }
      const float t2 = sum + t;                // Neumaier: keep the lost low part
      comp += fabsf(sum) >= fabsf(t) ? (sum - t2) + t : (t - t2) + sum;
      sum = t2;
    }
    red[threadIdx.x] = (double)sum + (double)comp;
    __syncthreads();
    for (int s2 = blockDim.x / 2; s2; s2 >>= 1) {
      if ((int)threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
      __syncthreads();
    }
    if (threadIdx.x == 0) marg_out[Pb.marg_off + o] = ldexp(red[0], -S.k);
    __syncthreads();
  }
}

cudaError_t launch_recombine(const DevPlan& p, const DevRes& r, int precision, const RecombSizes& z,
                             float* scratch, double* marg_out, double* zexp_out, cudaStream_t s) {
  auto grid = [](long long n, int per) {
    long long b = (n + per - 1) / per;
    return (unsigned)(b < 65535ll * 16 ? (b > 0 ? b : 1) : 65535ll * 16);
  };
  cudaError_t err = cudaSuccess;
  if (z.out_total > 0 && z.chain) {
    const bool use_tc = precision == CCS_BF16 && z.tensor_cores && z.rt_scratch && r.TQh && z.krange.full();
    // launch the R builder and the tiled GEMM only when some problem uses them
    // (a first-leaf problem builds its own table; streamed hubs have their own GEMM)
    bool need_r = false, need_gemm = false;
    for (int i = 0; i < z.n_problems; ++i) {
      const ProblemDev& Pb = z.host_problems[i];
      if (Pb.direct || Pb.general) continue;
      const bool tc = use_tc && Pb.tc;
      need_r = need_r || tc || !fact_path(Pb, precision, z.stitched, z.krange.full());
      need_gemm = need_gemm || (!tc && !Pb.stream);
    }
    if (z.r_total > 0 && need_r) {
      build_r_kernel<<<grid(z.r_total, 256), 256, 0, s>>>(p, r, precision, z.r_prefix, p.n_problems, z.r_total,
                                                          scratch, use_tc ? z.rt_scratch : nullptr, z.stitched,
                                                          z.krange.full() ? 1 : 0);
      note_launch();
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if (z.gemm_blocks > 0 && need_gemm) {
      if (z.max_tile_smem > 48 * 1024) {
        err = cudaFuncSetAttribute(gemm_splitk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, z.max_tile_smem);
        if (err != cudaSuccess) return err;
      }
      gemm_splitk_kernel<<<(unsigned)(z.gemm_blocks < 65535ll * 16 ? z.gemm_blocks : 65535ll * 16), 256,
                           z.max_tile_smem, s>>>(p, r, precision, z.blk_prefix, p.n_problems, z.gemm_blocks, scratch,
                                                 use_tc ? 1 : 0, z.krange); note_launch();
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    for (int i = 0; i < z.n_problems; ++i) {     // wide hubs off the tensor cores: streaming GEMM
      const ProblemDev& Pb = z.host_problems[i];
      if (!Pb.stream || Pb.direct || (use_tc && Pb.tc)) continue;
      if (fact_path(Pb, precision, z.stitched, z.krange.full())) {
        if ((err = launch_fact(p, r, Pb, scratch, s)) != cudaSuccess) return err;
        continue;
      }
      if ((err = launch_stream(r, Pb, scratch, precision == CCS_BF16 ? 1 : 0, z.stitched, z.krange, s)) !=
          cudaSuccess)
        return err;
    }
    if (use_tc) {
      for (int i = 0; i < z.n_problems; ++i) {
        const ProblemDev& Pb = z.host_problems[i];
        if (!Pb.tc) continue;
        {
          const long long tiles = ((Pb.K + 63) / 64) * ((Pb.M + 63) / 64);
          hub_bf16_kernel<<<(unsigned)(tiles < 152 * 32 ? tiles : 152 * 32), 256, 0, s>>>(
              hub_host_view(r, Pb), reinterpret_cast<__nv_bfloat16*>(r.TQh) + Pb.hub_T_off, Pb.M, Pb.K); note_launch();
          if ((err = cudaGetLastError()) != cudaSuccess) return err;
        }
        err = launch_gemm_tc(r.TQh + Pb.hub_T_off, z.rt_scratch + Pb.rt_off, Pb.M, Pb.N, Pb.K, Pb.splits,
                             scratch + Pb.part_off, r.status, s);
        if (err != cudaSuccess) return err;
      }
    }
    {
      reduce_scatter_kernel<<<grid(z.out_total, 32), 256, 0, s>>>(p, z.out_prefix, p.n_problems, z.out_total,
                                                                  scratch, marg_out, use_tc ? 1 : 0); note_launch();
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
  }
  if (z.has_general && z.out_total > 0) {
    general_contract_kernel<<<(unsigned)(z.out_total < 65535ll * 16 ? z.out_total : 65535ll * 16), 256, 0, s>>>(
        p, r, precision, z.out_prefix, p.n_problems, z.out_total, marg_out, z.krange);
    note_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const long long blocks = z.n_direct + z.z_total;
  if (blocks > 0) {
    const size_t smem = (size_t)z.direct_stage_floats * 2 * 4;
    if (smem > 48 * 1024) {
      err = cudaFuncSetAttribute(contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
    }
    contract_kernel<<<(unsigned)(blocks < 65535ll * 16 ? blocks : 65535ll * 16), 512, smem, s>>>(
        p, r, precision, z.direct_items, z.n_direct, z.direct_stage_floats, z.z_prefix, p.n_problems, z.z_total,
        marg_out, zexp_out, z.krange);
    note_launch();
    err = cudaGetLastError();
  }
  return err;
}

}  // namespace ccs
