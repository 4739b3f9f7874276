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

}  // namespace

__global__ void fold_kernel(DevPlan P, DevRes R, EvalParams E, const long long* prefix, int nf,
                            long long total) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int f = find_seg(prefix, nf, g);
    const FragDev& F = P.frags[f];
    const long long loc = g - prefix[f];
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

__global__ void fold_z_kernel(DevPlan P, DevRes R, const long long* prefix, int nf, long long total) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int f = find_seg(prefix, nf, g);
    const FragDev& F = P.frags[f];
    const long long loc = g - prefix[f];
    const int S2 = 2 * F.n_slots;
    const int zi = (int)(loc >> S2), Pi = (int)(loc & ((1ll << S2) - 1));
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
    R.TZ[F.TZ_off + loc] = (float)acc;
  }
}

// Small-shape contraction: one thread per output o of a star (hub + leaves),
// FP32 products summed in FP32 over chunks of 64 cut terms, chunks summed in
// FP64.  BF16 mode rounds both GEMM operands (hub tensor and the leaves'
// Kronecker product) to bf16 first, as a bf16 tensor-core GEMM would.
__global__ void recombine_small_kernel(DevPlan P, DevRes R, int precision, const long long* prefix,
                                       int np, long long total) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int pi = find_seg(prefix, np, g);
    const ProblemDev& Pb = P.problems[pi];
    const long long o = g - prefix[pi];
    const FragDev& Hb = P.frags[Pb.frag0 + Pb.hub];
    const int k = Pb.k;
    int oh = 0;
    for (int j = 0; j < Hb.m; ++j) oh |= (int)((o >> Hb.marg_pos[j]) & 1) << j;
    // leaves carrying cuts, plus a scalar for fragments without cuts
    int lf[kMaxCuts], lo[kMaxCuts], nl = 0;
    float scal = 1.f;
    for (int l = 0; l < Pb.n_frags; ++l) {
      if (l == Pb.hub) continue;
      const FragDev& L = P.frags[Pb.frag0 + l];
      int x = 0;
      for (int j = 0; j < L.m; ++j) x |= (int)((o >> L.marg_pos[j]) & 1) << j;
      if (L.n_slots == 0) {
        scal *= R.T[L.T_off + x];
      } else if (nl < kMaxCuts) {
        lf[nl] = Pb.frag0 + l;
        lo[nl] = x;
        ++nl;
      }
    }
    const long long K = 1ll << (2 * k);
    const float* th = R.T + Hb.T_off + (long long)oh * K;
    double total_d = 0.0;
    for (long long P0 = 0; P0 < K; P0 += 64) {
      float acc = 0.f;
      const long long P1 = P0 + 64 < K ? P0 + 64 : K;
      for (long long Pp = P0; Pp < P1; ++Pp) {
        float rv = scal;
        for (int l = 0; l < nl; ++l) {
          const FragDev& L = P.frags[lf[l]];
          int pl = 0;
          for (int i = 0; i < L.n_slots; ++i) pl |= (int)((Pp >> (2 * L.slot_cut[i])) & 3) << (2 * i);
          rv *= R.T[L.T_off + ((long long)lo[l] << (2 * L.n_slots)) + pl];
        }
        float hv = th[Pp];
        if (precision == CCS_BF16) {
          rv = to_bf16f(rv);
          hv = to_bf16f(hv);
        }
        acc = fmaf(hv, rv, acc);
      }
      total_d += (double)acc;
    }
    R.marg[Pb.marg_off + o] = ldexp(total_d, -k);
  }
}

// <Z_S> = 2^-k sum_P prod_f T_f^S(P|f): one block per (problem, string).
__global__ void recombine_z_kernel(DevPlan P, DevRes R, const long long* prefix, int np, long long total) {
  __shared__ double red[256];
  for (long long g = blockIdx.x; g < total; g += gridDim.x) {
    const int pi = find_seg(prefix, np, g);
    const ProblemDev& Pb = P.problems[pi];
    const int zi = (int)(g - prefix[pi]);
    const long long K = 1ll << (2 * Pb.k);
    double part = 0.0;
    for (long long P0 = (long long)threadIdx.x * 64; P0 < K; P0 += (long long)blockDim.x * 64) {
      float acc = 0.f;
      const long long P1 = P0 + 64 < K ? P0 + 64 : K;
      for (long long Pp = P0; Pp < P1; ++Pp) {
        float t = 1.f;
        for (int l = 0; l < Pb.n_frags; ++l) {
          const FragDev& L = P.frags[Pb.frag0 + l];
          int pl = 0;
          for (int i = 0; i < L.n_slots; ++i) pl |= (int)((Pp >> (2 * L.slot_cut[i])) & 3) << (2 * i);
          t *= R.TZ[L.TZ_off + ((long long)zi << (2 * L.n_slots)) + pl];
        }
        acc += t;
      }
      part += (double)acc;
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) R.zexp[Pb.zexp_off + zi] = ldexp(red[0], -Pb.k);
    __syncthreads();
  }
}

cudaError_t launch_fold(const DevPlan& p, const DevRes& r, const EvalParams& e, const long long* t_prefix,
                        int nf, long long total, const long long* tz_prefix, long long total_z,
                        cudaStream_t s) {
  if (total > 0) {
    const long long blocks = (total + 255) / 256;
    fold_kernel<<<(unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8), 256, 0, s>>>(p, r, e, t_prefix, nf, total);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (total_z > 0) {
    const long long blocks = (total_z + 255) / 256;
    fold_z_kernel<<<(unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8), 256, 0, s>>>(p, r, tz_prefix, nf, total_z);
  }
  return cudaGetLastError();
}

cudaError_t launch_recombine(const DevPlan& p, const DevRes& r, int precision, const long long* out_prefix,
                             long long total_out, const long long* z_prefix, long long total_z,
                             cudaStream_t s) {
  if (total_out > 0) {
    const long long blocks = (total_out + 127) / 128;
    recombine_small_kernel<<<(unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8), 128, 0, s>>>(
        p, r, precision, out_prefix, p.n_problems, total_out);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (total_z > 0) {
    recombine_z_kernel<<<(unsigned)(total_z < 65535 ? total_z : 65535), 256, 0, s>>>(p, r, z_prefix, p.n_problems,
                                                                               total_z);
  }
  return cudaGetLastError();
}

}  // namespace ccs
