// Maximum-likelihood correction of fragment models (Sec. V-C: before the
// contraction the fragment data become self-consistent fragment models,
// which mitigates the sampling error of the Clifford fragments' shots).
//
// A fragment's model is its Choi form, one Hermitian operator per outcome o
// of its marginal wires on its d cut slots:
//   J_o = 2^-d sum_P T_f(o, P) (x)_j s_j(P_j),  s_j(P) = P^T at a quantum
//   input, P at a quantum output;  T_f(o, P) = Tr[(x)_j s_j(P_j) J_o].
// Physical: every J_o positive semidefinite, sum_o Tr J_o = 2^{q_in}.  The
// maximum-likelihood model under Gaussian shot noise of equal variance per
// T_f entry is the nearest physical one in Frobenius norm: all blocks'
// eigenvalues projected together onto {lambda >= 0, sum = 2^{q_in}}, each
// block rebuilt from its own eigenvectors (the eigenvalue projection of
// Smolin, Gambetta and Smith, PRL 108, 070502, 2012).
//
// GPU form, three launches per group of fragments with the same d (d <= 6):
//  1. ml_eig_kernel, one CTA per (fragment, outcome): the block's T_f row
//     (a star hub's operand is stored by preparation at its inputs and is
//     turned into Pauli digits first), the Choi block J_o (D = 2^d rows,
//     complex64, rows padded to D + 1 so that row and column sweeps are free
//     of bank conflicts), and a cyclic complex Jacobi eigendecomposition in
//     shared memory: D/2 disjoint rotations per round in the round-robin
//     order, D - 1 rounds per sweep, sweeps until no rotation is left above
//     2^-24 of the block's Frobenius norm (at most kMlMaxSweeps).  Each
//     rotation is a phase that makes the pair's off-diagonal entry real
//     followed by the real symmetric 2 x 2 Schur rotation (Golub & Van Loan,
//     Sec. 8.5).  The eigenvalues and eigenvectors go to a scratch array.
//  2. ml_threshold_kernel, one CTA per fragment: the threshold theta with
//     sum max(lambda - theta, 0) = 2^{q_in} over its eigenvalue list, by
//     Michelot's finite algorithm (J. Optim. Theory Appl. 50, 1986):
//     theta = (sum of the kept values - total) / (their count), keep the
//     values above theta, repeat until the kept set stops changing.
//  3. ml_rebuild_kernel, one CTA per (fragment, outcome): J'_o from the
//     eigenvectors with eigenvalues max(lambda - theta, 0), then T'_f(o, P);
//     written to T_f, and a hub's operand (by preparation at its inputs) is
//     rewritten in FP32.
#include "kernels.cuh"

namespace ccs {

namespace {

constexpr int kMlMaxSweeps = 30;

__device__ __forceinline__ int ml_find(const MlFrag* __restrict__ fr, int n, long long blk) {
  int lo = 0, hi = n;      // fr[lo].blk0 <= blk < fr[hi].blk0
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (fr[mid].blk0 <= blk) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Sum over the CTA (every thread gets the result); red holds 32 entries.
template <class T>
__device__ T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  T s = 0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Largest value over the CTA (every thread gets it); red holds 32 entries.
__device__ float block_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  float m = 0.f;
  for (int i = 0; i < nw; ++i) m = fmaxf(m, red[i]);
  return m;
}

// Entry [r][c] of the slot operator (x)_j s_j(P_j) for the Pauli digits of P
// where the entry is nonzero: returns the power of i (0..3) of the entry
// (its value is i^pw, a sign folded in as 2).  At slot j the entry needs
// P_j in {I, Z} when r_j == c_j and in {X, Y} otherwise; Z contributes
// (-1)^{r_j}; Y at an output contributes -i for r_j = 0 and +i for r_j = 1,
// its transpose at an input the opposite.
__device__ __forceinline__ int slot_entry_phase(int P, int r, int d, unsigned inmask) {
  int pw = 0;
  for (int j = 0; j < d; ++j) {
    const int pj = (P >> (2 * j)) & 3, rj = (r >> j) & 1;
    if (pj == 3) pw += 2 * rj;
    else if (pj == 2) pw += 1 + 2 * ((rj ^ 1) ^ (int)((inmask >> j) & 1));
  }
  return pw & 3;
}

__device__ __forceinline__ unsigned input_mask(const FragDev& F) {
  unsigned m = 0;
  for (int j = 0; j < F.n_slots; ++j)
    if ((F.slot_code[j] >> 8) == 0) m |= 1u << j;
  return m;
}

}  // namespace

// One CTA per (fragment, outcome o) of a group with d cut slots.
__global__ void __launch_bounds__(256, 3) ml_eig_kernel(DevPlan P, DevRes R, const MlFrag* __restrict__ fr,
                                                        int nfr, int d, float* __restrict__ scratch) {
  extern __shared__ __align__(16) float2 smc[];
  const int D = 1 << d, LD = D + 1, KP = 1 << (2 * d), H = D / 2;
  float2* A = smc;               // D x LD: the Choi block, then its rotations
  float2* V = A + D * LD;        // D x LD: the accumulated unitary, transposed (row k = column k of V)
  float* sT = reinterpret_cast<float*>(V);   // the block's T_f row (4^d), before V is set up
  float4* prm = reinterpret_cast<float4*>(V + D * LD);   // per pair: (c, s, t, Re w), (Im w, a_pp, a_qq, |a_pq|)
  int2* pq = reinterpret_cast<int2*>(prm + 2 * H);        // per pair: p, q
  int* blk_ij = reinterpret_cast<int*>(pq + H);           // pair blocks i <= j of a round: i | j << 16
  __shared__ float red[32];
  __shared__ int any_rot;
  const int tid = threadIdx.x, nt = blockDim.x;

  const long long blk = blockIdx.x;
  const MlFrag& mf = fr[ml_find(fr, nfr, blk)];
  const FragDev& F = P.frags[mf.frag];
  const int o = (int)(blk - mf.blk0);
  const unsigned inmask = input_mask(F);

  // 1. the block's row of T_f
  if (!mf.hub) {
    const float* src = R.T + F.T_off + ((long long)o << (2 * d));
    for (int i = tid; i < KP; i += nt) sT[i] = src[i];
  } else {   // hub operand Q^T[D][o]: preparation digit s at each input slot
    const long long Mo = 1ll << F.m;
    if (mf.i16) {
      const int16_t* q = reinterpret_cast<const int16_t*>(R.TQ + F.T_off);
      for (int i = tid; i < KP; i += nt) sT[i] = (float)q[(long long)i * Mo + o] * R.hub_scale;
    } else {
      for (int i = tid; i < KP; i += nt) sT[i] = R.TQ[F.T_off + (long long)i * Mo + o];
    }
    // T(P_j) = sum_s mu(P_j, s) Q(s): I = Q0 + Q1, X = 2 Q2 - Q0 - Q1,
    // Y = 2 Q3 - Q0 - Q1, Z = Q0 - Q1 (the prepared states |0>,|1>,|+>,|+i>)
    for (int j = 0; j < d; ++j) {
      if (!((inmask >> j) & 1)) continue;
      __syncthreads();
      const int st = 1 << (2 * j);
      for (int g = tid; g < KP / 4; g += nt) {
        const int b = ((g >> (2 * j)) << (2 * j + 2)) | (g & (st - 1));
        const float q0 = sT[b], q1 = sT[b + st], q2 = sT[b + 2 * st], q3 = sT[b + 3 * st];
        sT[b] = q0 + q1;
        sT[b + st] = 2.f * q2 - q0 - q1;
        sT[b + 2 * st] = 2.f * q3 - q0 - q1;
        sT[b + 3 * st] = q0 - q1;
      }
    }
  }
  __syncthreads();

  // 2. J_o[r][c] = 2^-d sum over the 2^d Paulis whose slot operator is
  //    nonzero at [r][c]
  const float scale = 1.f / (float)D;
  float nrm = 0.f;
  for (int e = tid; e < D * D; e += nt) {
    const int r = e >> d, c = e & (D - 1), x = r ^ c;
    float re = 0.f, im = 0.f;
    for (int t = 0; t < D; ++t) {
      int Pi = 0;
      for (int j = 0; j < d; ++j) {
        const int xj = (x >> j) & 1, tj = (t >> j) & 1;
        Pi |= (xj ? (tj ? 2 : 1) : (tj ? 3 : 0)) << (2 * j);
      }
      const float v = sT[Pi];
      switch (slot_entry_phase(Pi, r, d, inmask)) {
        case 0: re += v; break;
        case 1: im += v; break;
        case 2: re -= v; break;
        default: im -= v; break;
      }
    }
    re *= scale;
    im *= scale;
    A[r * LD + c] = make_float2(re, im);
    nrm += re * re + im * im;
  }
  nrm = block_sum(nrm, red);     // its barriers also end the reads of sT
  for (int e = tid; e < D * D; e += nt) {
    const int r = e >> d, c = e & (D - 1);
    V[r * LD + c] = make_float2(r == c ? 1.f : 0.f, 0.f);
  }
  const float tol = sqrtf(nrm) * 5.9604645e-8f;   // 2^-24 of the Frobenius norm
  for (int j = tid; j < H; j += nt)
    for (int i = 0; i <= j; ++i) blk_ij[j * (j + 1) / 2 + i] = i | (j << 16);

  // 3. cyclic Jacobi, round-robin pairs: round t pairs (D-1, t) and
  //    ((t + i) mod (D-1), (t - i) mod (D-1)) for i = 1 .. D/2 - 1.  With
  //    a_pq = |a_pq| w, the rotation U = [[c, s], [-s conj(w), c conj(w)]]
  //    on columns (p, q) zeroes a_pq and leaves a_pp - t |a_pq|,
  //    a_qq + t |a_pq| on the diagonal.  All of a round's rotations are
  //    applied at once, A <- U^H A U block by block: the 2 x 2 block of pairs
  //    (i, j), i < j, becomes U_i^H B U_j and its mirror block the conjugate
  //    transpose (so A stays exactly Hermitian); V^T's rows p, q take the
  //    column update of V <- V U.
  if (nrm > 0.f && D > 1) {
    const int nblk = H * (H + 1) / 2;
    const int lg_tpp = max(0, (31 - __clz(nt)) - (d - 1));   // threads per pair in the V^T update
    const int vi = tid >> lg_tpp, vl = tid & ((1 << lg_tpp) - 1);
    for (int sweep = 0; sweep < kMlMaxSweeps; ++sweep) {
      if (tid == 0) any_rot = 0;
      __syncthreads();
      for (int t = 0; t < D - 1; ++t) {
        if (tid < H) {
          int a, b;
          if (tid == 0) { a = D - 1; b = t; }
          else { a = (t + tid) % (D - 1); b = (t - tid + D - 1) % (D - 1); }
          const int p = min(a, b), q = max(a, b);
          const float app = A[p * LD + p].x, aqq = A[q * LD + q].x;
          const float2 apq = A[p * LD + q];
          const float mag = sqrtf(apq.x * apq.x + apq.y * apq.y);
          float c = 1.f, s = 0.f, tt = 0.f, wr = 1.f, wi = 0.f;
          if (mag > tol) {
            const float tau = (aqq - app) / (2.f * mag);
            tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = 1.f / sqrtf(1.f + tt * tt);
            s = tt * c;
            wr = apq.x / mag;
            wi = apq.y / mag;
            if (tt != 0.f) any_rot = 1;
          }
          prm[2 * tid] = make_float4(c, s, tt, wr);
          prm[2 * tid + 1] = make_float4(wi, app, aqq, mag);
          pq[tid] = make_int2(p, q);
        }
        __syncthreads();
        // A: one 2 x 2 block per pair of pairs (i <= j)
        for (int e = tid; e < nblk; e += nt) {
          const int ij = blk_ij[e], i = ij & 0xffff, j = ij >> 16;
          const float4 pi0 = prm[2 * i], pj0 = prm[2 * j];
          const bool ri = pi0.z != 0.f, rj = pj0.z != 0.f;
          if (!ri && !rj) continue;
          const float4 pi1 = prm[2 * i + 1];
          const int2 pqi = pq[i];
          const int p = pqi.x, q = pqi.y;
          if (i == j) {
            A[p * LD + p] = make_float2(pi1.y - pi0.z * pi1.w, 0.f);
            A[q * LD + q] = make_float2(pi1.z + pi0.z * pi1.w, 0.f);
            A[p * LD + q] = make_float2(0.f, 0.f);
            A[q * LD + p] = make_float2(0.f, 0.f);
            continue;
          }
          const float4 pj1 = prm[2 * j + 1];
          const int2 pqj = pq[j];
          const int u = pqj.x, v = pqj.y;
          float2 b00 = A[p * LD + u], b01 = A[p * LD + v], b10 = A[q * LD + u], b11 = A[q * LD + v];
          if (rj) {   // B <- B U_j: columns c b0 - s conj(w) b1, s b0 + c conj(w) b1
            const float c = pj0.x, s = pj0.y, wr = pj0.w, wi = -pj1.x;
            const float2 y0 = make_float2(wr * b01.x - wi * b01.y, wr * b01.y + wi * b01.x);
            const float2 y1 = make_float2(wr * b11.x - wi * b11.y, wr * b11.y + wi * b11.x);
            const float2 n00 = make_float2(c * b00.x - s * y0.x, c * b00.y - s * y0.y);
            const float2 n01 = make_float2(s * b00.x + c * y0.x, s * b00.y + c * y0.y);
            const float2 n10 = make_float2(c * b10.x - s * y1.x, c * b10.y - s * y1.y);
            const float2 n11 = make_float2(s * b10.x + c * y1.x, s * b10.y + c * y1.y);
            b00 = n00; b01 = n01; b10 = n10; b11 = n11;
          }
          if (ri) {   // B <- U_i^H B: rows c r0 - s w r1, s r0 + c w r1
            const float c = pi0.x, s = pi0.y, wr = pi0.w, wi = pi1.x;
            const float2 y0 = make_float2(wr * b10.x - wi * b10.y, wr * b10.y + wi * b10.x);
            const float2 y1 = make_float2(wr * b11.x - wi * b11.y, wr * b11.y + wi * b11.x);
            const float2 n00 = make_float2(c * b00.x - s * y0.x, c * b00.y - s * y0.y);
            const float2 n01 = make_float2(c * b01.x - s * y1.x, c * b01.y - s * y1.y);
            const float2 n10 = make_float2(s * b00.x + c * y0.x, s * b00.y + c * y0.y);
            const float2 n11 = make_float2(s * b01.x + c * y1.x, s * b01.y + c * y1.y);
            b00 = n00; b01 = n01; b10 = n10; b11 = n11;
          }
          A[p * LD + u] = b00; A[p * LD + v] = b01; A[q * LD + u] = b10; A[q * LD + v] = b11;
          A[u * LD + p] = make_float2(b00.x, -b00.y);
          A[v * LD + p] = make_float2(b01.x, -b01.y);
          A[u * LD + q] = make_float2(b10.x, -b10.y);
          A[v * LD + q] = make_float2(b11.x, -b11.y);
        }
        // V^T rows p, q (one pair per group of threads, its rotation in registers)
        if (vi < H) {
          const float4 pr0 = prm[2 * vi];
          if (pr0.z != 0.f) {
            const int2 pqv = pq[vi];
            const int p = pqv.x, q = pqv.y;
            const float c = pr0.x, s = pr0.y, wr = pr0.w, wi = -prm[2 * vi + 1].x;
            for (int r = vl; r < D; r += (1 << lg_tpp)) {
              const float2 vp = V[p * LD + r], vq = V[q * LD + r];
              const float2 y = make_float2(wr * vq.x - wi * vq.y, wr * vq.y + wi * vq.x);
              V[p * LD + r] = make_float2(c * vp.x - s * y.x, c * vp.y - s * y.y);
              V[q * LD + r] = make_float2(s * vp.x + c * y.x, s * vp.y + c * y.y);
            }
          }
        }
        __syncthreads();
      }
      // stop once no off-diagonal entry exceeds the tolerance (the next
      // sweep would rotate nothing)
      float off = 0.f;
      for (int e2 = tid; e2 < D * D; e2 += nt) {
        const int r = e2 >> d, c = e2 & (D - 1);
        if (r != c) {
          const float2 x = A[r * LD + c];
          off = fmaxf(off, x.x * x.x + x.y * x.y);
        }
      }
      off = block_max(off, red);
      const int more = any_rot;
      __syncthreads();
      if (!more || off <= tol * tol) break;
    }
  }
  __syncthreads();

  // 4. eigenvalues (the real diagonal) and eigenvectors (the rows of V^T,
  //    stored row-major D x D complex: entry [k][r] = component r of vector k)
  float* ev = scratch + mf.ev_off + (long long)o * D;
  float2* vec = reinterpret_cast<float2*>(scratch + mf.vec_off) + (long long)o * D * D;
  for (int i = tid; i < D; i += nt) ev[i] = A[i * LD + i].x;
  for (int e = tid; e < D * D; e += nt) vec[e] = V[(e >> d) * LD + (e & (D - 1))];
}

// One CTA per fragment: theta over its eigenvalue list.
__global__ void __launch_bounds__(256) ml_threshold_kernel(DevPlan P, const MlFrag* __restrict__ fr,
                                                           const float* __restrict__ scratch,
                                                           double* __restrict__ theta_out) {
  __shared__ double redd[32];
  __shared__ long long redc[32];
  const MlFrag& mf = fr[blockIdx.x];
  const FragDev& F = P.frags[mf.frag];
  const long long n = (1ll << F.m) << mf.d;
  const float* ev = scratch + mf.ev_off;
  double theta = -1e300;
  long long prev = -1;
  // the kept set only shrinks, so at most n + 1 passes; the cap bounds the
  // loop should rounding ever make it oscillate
  for (long long it = 0; it <= n + 1 && it < 4096; ++it) {
    double s = 0.0;
    long long cnt = 0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = ev[i];
      if (v > theta) { s += v; ++cnt; }
    }
    s = block_sum(s, redd);
    cnt = block_sum(cnt, redc);
    if (cnt == prev || cnt == 0) break;
    prev = cnt;
    const double th = (s - mf.total) / (double)cnt;
    theta = th > theta ? th : theta;
  }
  if (threadIdx.x == 0) theta_out[blockIdx.x] = theta;
}

// One CTA per (fragment, outcome o): the corrected block and T'_f row.
__global__ void __launch_bounds__(256) ml_rebuild_kernel(DevPlan P, DevRes R, const MlFrag* __restrict__ fr,
                                                         int nfr, int d, const float* __restrict__ scratch,
                                                         const double* __restrict__ theta) {
  extern __shared__ float2 smc[];
  const int D = 1 << d, LD = D + 1, KP = 1 << (2 * d);
  float2* V = smc;               // D x LD eigenvectors (row k = vector k)
  float2* J = V + D * LD;        // D x LD: J'
  float* lam = reinterpret_cast<float*>(J + D * LD);   // D clipped eigenvalues
  float* sT = lam + D;           // 4^d
  int* live = reinterpret_cast<int*>(sT + KP);          // indices of the nonzero eigenvalues
  __shared__ int n_live;
  const int tid = threadIdx.x, nt = blockDim.x;

  const long long blk = blockIdx.x;
  const MlFrag& mf = fr[ml_find(fr, nfr, blk)];
  const FragDev& F = P.frags[mf.frag];
  const int o = (int)(blk - mf.blk0);
  const unsigned inmask = input_mask(F);
  const float th = (float)theta[mf.index];
  const float* ev = scratch + mf.ev_off + (long long)o * D;
  const float2* vec = reinterpret_cast<const float2*>(scratch + mf.vec_off) + (long long)o * D * D;
  for (int e = tid; e < D * D; e += nt) V[(e >> d) * LD + (e & (D - 1))] = vec[e];
  for (int i = tid; i < D; i += nt) lam[i] = fmaxf(ev[i] - th, 0.f);
  __syncthreads();
  if (tid == 0) {
    int k = 0;
    for (int i = 0; i < D; ++i)
      if (lam[i] > 0.f) live[k++] = i;
    n_live = k;
  }
  __syncthreads();
  const int nl = n_live;
  // J'[r][c] = sum_k lam_k v_k[r] conj(v_k[c])
  for (int e = tid; e < D * D; e += nt) {
    const int r = e >> d, c = e & (D - 1);
    float re = 0.f, im = 0.f;
    for (int t = 0; t < nl; ++t) {
      const int k = live[t];
      const float l = lam[k];
      const float2 a = V[k * LD + r], b = V[k * LD + c];
      re += l * (a.x * b.x + a.y * b.y);
      im += l * (a.y * b.x - a.x * b.y);
    }
    J[r * LD + c] = make_float2(re, im);
  }
  __syncthreads();
  // T'(P) = Re Tr[S_P J'] = sum_r Re(S_P[r][c] J'[c][r]), c = r xor x(P)
  for (int Pi = tid; Pi < KP; Pi += nt) {
    int x = 0;
    for (int j = 0; j < d; ++j) {
      const int pj = (Pi >> (2 * j)) & 3;
      if (pj == 1 || pj == 2) x |= 1 << j;
    }
    float acc = 0.f;
    for (int r = 0; r < D; ++r) {
      const float2 v = J[(r ^ x) * LD + r];
      switch (slot_entry_phase(Pi, r, d, inmask)) {   // Re(i^pw (re + i im))
        case 0: acc += v.x; break;
        case 1: acc -= v.y; break;
        case 2: acc -= v.x; break;
        default: acc += v.y; break;
      }
    }
    sT[Pi] = acc;
  }
  __syncthreads();
  float* dst = R.T + F.T_off + ((long long)o << (2 * d));
  for (int i = tid; i < KP; i += nt) dst[i] = sT[i];
  if (!mf.hub) return;
  // the hub's operand by preparation at its inputs: Q(s) = Tr[E(rho_s) ...]
  // = (T_I + T_Z)/2, (T_I - T_Z)/2, (T_I + T_X)/2, (T_I + T_Y)/2
  for (int j = 0; j < d; ++j) {
    if (!((inmask >> j) & 1)) continue;
    __syncthreads();
    const int st = 1 << (2 * j);
    for (int g = tid; g < KP / 4; g += nt) {
      const int b = ((g >> (2 * j)) << (2 * j + 2)) | (g & (st - 1));
      const float tI = sT[b], tX = sT[b + st], tY = sT[b + 2 * st], tZ = sT[b + 3 * st];
      sT[b] = 0.5f * (tI + tZ);
      sT[b + st] = 0.5f * (tI - tZ);
      sT[b + 2 * st] = 0.5f * (tI + tX);
      sT[b + 3 * st] = 0.5f * (tI + tY);
    }
  }
  __syncthreads();
  const long long Mo = 1ll << F.m;
  for (int i = tid; i < KP; i += nt) R.TQ[F.T_off + (long long)i * Mo + o] = sT[i];
}

size_t ml_eig_smem(int d) {
  const size_t D = 1u << d, LD = D + 1, KP = 1u << (2 * d), H = D / 2;
  const size_t v_floats = 2 * D * LD > KP ? 2 * D * LD : KP;   // V shares its space with the T_f row
  return 2 * D * LD * sizeof(float) + v_floats * sizeof(float) + 8 * (H + 1) * sizeof(float) +
         2 * (H + 1) * sizeof(int) + (H * (H + 1) / 2 + 1) * sizeof(int);
}
size_t ml_rebuild_smem(int d) {
  const size_t D = 1u << d, LD = D + 1, KP = 1u << (2 * d);
  return (4 * D * LD + D + KP + D) * sizeof(float);
}

cudaError_t launch_ml_correct(const DevPlan& p, const DevRes& r, const MlFrag* d_frags, int n_frags,
                              const MlGroup* groups, int n_groups, float* scratch, double* theta, cudaStream_t s) {
  cudaError_t err;
  for (int g = 0; g < n_groups; ++g) {
    const MlGroup& G = groups[g];
    const size_t sm = ml_eig_smem(G.d);
    if ((err = cudaFuncSetAttribute(ml_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
        cudaSuccess)
      return err;
    const int threads = G.d >= 4 ? 256 : 64;
    ml_eig_kernel<<<(unsigned)G.blocks, threads, sm, s>>>(p, r, d_frags + G.first, G.count, G.d, scratch);
    note_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  ml_threshold_kernel<<<n_frags, 256, 0, s>>>(p, d_frags, scratch, theta);
  note_launch();
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  for (int g = 0; g < n_groups; ++g) {
    const MlGroup& G = groups[g];
    const size_t sm = ml_rebuild_smem(G.d);
    if ((err = cudaFuncSetAttribute(ml_rebuild_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
        cudaSuccess)
      return err;
    const int threads = G.d >= 4 ? 256 : 64;
    ml_rebuild_kernel<<<(unsigned)G.blocks, threads, sm, s>>>(p, r, d_frags + G.first, G.count, G.d, scratch,
                                                               theta);
    note_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace ccs
