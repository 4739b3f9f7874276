// Clifford-fragment kernels: bit-packed CHP tableau evolution (K1), reduction
// to the canonical affine outcome space (K2), Z-string values (K7 inputs) and
// Philox shot sampling (K3).
//
// Tableau layout in shared memory (one variant per CTA): column-major,
// bit-sliced over rows.  Columns X_0..X_n (X_n is an all-zero dummy used as
// the second operand of one-qubit ops), Z_0..Z_n, then the sign column R;
// each column holds W = 2*Wh uint64 words: destabilizer rows 0..n-1 in words
// [0, Wh), stabilizer rows in words [Wh, 2Wh), so destabilizer i and
// stabilizer i share a bit position.  A gate therefore touches whole 64-row
// words of a few columns (Gottesman-Knill / CHP, Sec. II-C and III-B).
#include "kernels.cuh"

namespace ccs {

constexpr int kMaxWh = (kMaxTableauQubits + 63) / 64;

namespace {

__device__ __forceinline__ uint64_t bm(unsigned v, int bit) { return 0ull - (uint64_t)((v >> bit) & 1u); }

// Apply one fused Clifford op to word w of its four columns.
__device__ __forceinline__ void apply_op(CliffordOp op, uint64_t* tab, int W, int zb, int w,
                                         uint64_t& rdelta) {
  uint64_t* pxa = tab + (size_t)op.qa * W + w;
  uint64_t* pza = tab + (size_t)(zb + op.qa) * W + w;
  uint64_t* pxb = tab + (size_t)op.qb * W + w;
  uint64_t* pzb = tab + (size_t)(zb + op.qb) * W + w;
  const uint64_t v0 = *pxa, v1 = *pza, v2 = *pxb, v3 = *pzb;
  const unsigned M = op.M, A = op.anf;
  const uint64_t u0 = (v0 & bm(M, 0)) ^ (v1 & bm(M, 1)) ^ (v2 & bm(M, 2)) ^ (v3 & bm(M, 3));
  const uint64_t u1 = (v0 & bm(M, 4)) ^ (v1 & bm(M, 5)) ^ (v2 & bm(M, 6)) ^ (v3 & bm(M, 7));
  const uint64_t u2 = (v0 & bm(M, 8)) ^ (v1 & bm(M, 9)) ^ (v2 & bm(M, 10)) ^ (v3 & bm(M, 11));
  const uint64_t u3 = (v0 & bm(M, 12)) ^ (v1 & bm(M, 13)) ^ (v2 & bm(M, 14)) ^ (v3 & bm(M, 15));
  const uint64_t v01 = v0 & v1, v23 = v2 & v3;
  uint64_t f = (v0 & bm(A, 1)) ^ (v1 & bm(A, 2)) ^ (v01 & bm(A, 3)) ^ (v2 & bm(A, 4)) ^
               ((v0 & v2) & bm(A, 5)) ^ ((v1 & v2) & bm(A, 6)) ^ ((v01 & v2) & bm(A, 7)) ^
               (v3 & bm(A, 8)) ^ ((v0 & v3) & bm(A, 9)) ^ ((v1 & v3) & bm(A, 10)) ^
               ((v01 & v3) & bm(A, 11)) ^ (v23 & bm(A, 12)) ^ ((v0 & v23) & bm(A, 13)) ^
               ((v1 & v23) & bm(A, 14)) ^ ((v01 & v23) & bm(A, 15));
  rdelta ^= f;
  *pxa = u0;
  *pza = u1;
  *pxb = u2;
  *pzb = u3;
}

// XOR of the bits strictly below each position.
__device__ __forceinline__ uint64_t prefix_xor_excl(uint64_t x) {
  uint64_t p = x << 1;
  p ^= p << 1;
  p ^= p << 2;
  p ^= p << 4;
  p ^= p << 8;
  p ^= p << 16;
  p ^= p << 32;
  return p;
}

// <Z_Q> of the stabilizer state for the wire set Q, given per lane w the
// XOR over q in Q of column X_q word w (acc; 0 on lanes >= W).  Z_Q
// anticommutes with a stabilizer -> 0.  Otherwise Z_Q = +-prod_{i in S} stab_i
// with S the destabilizers anticommuting with Z_Q; the sign is found by
// multiplying those rows in index order, per qubit, with the phase of each
// single-qubit product counted by popcounts (mod 4).  Warp-cooperative;
// `sel` is this warp's scratch of >= Wh words.
__device__ int zexp_from_acc(const uint64_t* tab, int n, int W, int Wh, uint64_t acc, int lane,
                             uint64_t* sel, unsigned* bad) {
  const unsigned FULL = 0xffffffffu;
  const bool anti = __any_sync(FULL, lane >= Wh && lane < W && acc != 0);
  if (anti) return 0;
  if (lane < Wh) sel[lane] = acc;
  __syncwarp();
  const int zb = n + 1;
  int e = 0;
  unsigned xres = 0;
  for (int j = lane; j < n; j += 32) {
    unsigned cx = 0, cz = 0;
    for (int w = 0; w < Wh; ++w) {
      const uint64_t s = sel[w];
      if (s == 0) continue;
      const uint64_t x = tab[(size_t)j * W + Wh + w] & s;
      const uint64_t z = tab[(size_t)(zb + j) * W + Wh + w] & s;
      const uint64_t px = prefix_xor_excl(x) ^ (cx ? ~0ull : 0ull);
      const uint64_t pz = prefix_xor_excl(z) ^ (cz ? ~0ull : 0ull);
      const uint64_t X1 = px & ~pz, Y1 = px & pz, Z1 = ~px & pz;
      const uint64_t X2 = x & ~z, Y2 = x & z, Z2 = ~x & z;
      const uint64_t plus = (X1 & Y2) | (Y1 & Z2) | (Z1 & X2);
      const uint64_t minus = (X1 & Z2) | (Y1 & X2) | (Z1 & Y2);
      e += __popcll(plus) - __popcll(minus);
      cx ^= __popcll(x) & 1;
      cz ^= __popcll(z) & 1;
    }
    xres |= cx;
  }
  // signs of the selected stabilizers
  if (lane < Wh) e += 2 * __popcll(tab[(size_t)(2 * (n + 1)) * W + Wh + lane] & sel[lane]);
  for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(FULL, e, o);
  const bool xleft = __any_sync(FULL, xres != 0);
  __syncwarp();
  const int ph = ((e % 4) + 4) % 4;
  if ((ph & 1) || xleft) {
    if (lane == 0) atomicOr(bad, 1u);
    return 0;
  }
  return ph == 2 ? -1 : 1;
}

__device__ __forceinline__ int variant_in_digit(int v, int i) {
  for (int t = 0; t < i; ++t) v /= 4;
  return v % 4;
}
__device__ __forceinline__ int variant_out_digit(int v, int qin, int i) {
  for (int t = 0; t < qin; ++t) v /= 4;
  for (int t = 0; t < i; ++t) v /= 3;
  return v % 3;
}

}  // namespace

__global__ void __launch_bounds__(512) clifford_kernel(DevPlan P, DevRes R, EvalParams E) {
  extern __shared__ unsigned long long smem_u64[];
  uint64_t* tab = reinterpret_cast<uint64_t*>(smem_u64);
  __shared__ int s_item;
  __shared__ int s_rank;
  __shared__ uint32_t s_off;
  __shared__ uint32_t s_basis[kMaxMeas];
  __shared__ int s_piv[kMaxMeas];
  __shared__ uint32_t s_nonpiv_mask[kMaxMeas];   // pivots whose basis row has bit j
  __shared__ int s_nonpiv[kMaxMeas];
  __shared__ int s_n_nonpiv;
  __shared__ uint64_t s_sel[16][kMaxWh];

  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;

  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(&R.work[0], 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= P.n_items_cliff) break;
    const int2 it = P.items_cliff[item];
    const FragDev& F = P.frags[it.x];
    const int v = it.y;
    const int n = F.n, W = F.W, Wh = F.Wh, zb = n + 1, rcol = 2 * (n + 1);
    const int ncol = 2 * n + 3;
    uint32_t* rows = reinterpret_cast<uint32_t*>(tab + (size_t)ncol * W);

    // --- K1: initial tableau (destabilizer i = X_i, stabilizer i = Z_i) ---
    for (int i = tid; i < ncol * W; i += nt) tab[i] = 0ull;
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      tab[(size_t)j * W + (j >> 6)] = 1ull << (j & 63);
      tab[(size_t)(zb + j) * W + Wh + (j >> 6)] = 1ull << (j & 63);
    }
    __syncthreads();

    const int J = nt / W;                  // op slots per word
    const int w = tid % W, jslot = tid / W;
    const bool active = jslot < J;
    uint64_t rdelta = 0;
    if (active) {                          // preparations at quantum inputs
      for (int o = jslot; o < F.qin; o += J) {
        CliffordOp op = P.prep_ops[variant_in_digit(v, o)];
        op.qa = (uint16_t)P.wires[F.qin_off + o];
        op.qb = (uint16_t)n;
        apply_op(op, tab, W, zb, w, rdelta);
      }
    }
    __syncthreads();
    for (int mm = 0; mm < F.n_moments; ++mm) {
      const int b0 = P.moments[F.mom_off + mm], b1 = P.moments[F.mom_off + mm + 1];
      if (active)
        for (int o = b0 + jslot; o < b1; o += J) apply_op(P.cops[F.ops_off + o], tab, W, zb, w, rdelta);
      __syncthreads();
    }
    if (active) {                          // basis changes at quantum outputs
      for (int o = jslot; o < F.qout; o += J) {
        CliffordOp op = P.basis_ops[variant_out_digit(v, F.qin, o)];
        op.qa = (uint16_t)P.wires[F.qout_off + o];
        op.qb = (uint16_t)n;
        apply_op(op, tab, W, zb, w, rdelta);
      }
      atomicXor(reinterpret_cast<unsigned long long*>(&tab[(size_t)rcol * W + w]),
                (unsigned long long)rdelta);
    }
    __syncthreads();

    if (E.keep_tableaus && F.tab_off >= 0) {
      unsigned long long* dst = R.tabs + F.tab_off + (long long)v * ncol * W;
      for (int i = tid; i < ncol * W; i += nt) dst[i] = tab[i];
    }

    // --- K2: basis B = RREF of the stabilizer X-block on the columns A ---
    const int nA = F.nA;
    for (int i = tid; i < n; i += nt) {
      uint32_t row = 0;
      for (int j = 0; j < nA; ++j) {
        const int a = P.wires[F.A_off + j];
        row |= (uint32_t)((tab[(size_t)a * W + Wh + (i >> 6)] >> (i & 63)) & 1ull) << j;
      }
      rows[i] = row;
    }
    if (tid == 0) s_off = 0;
    __syncthreads();
    if (warp == 0) {
      int cnt = 0;
      for (int p = 0; p < nA; ++p) {
        int cand = 0x7fffffff;
        for (int i = lane; i < n; i += 32)
          if ((rows[i] >> p) & 1u) { cand = i; break; }
        for (int o = 16; o; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
        if (cand == 0x7fffffff) continue;
        const uint32_t prow = rows[cand];
        __syncwarp();
        if (lane == 0) rows[cand] = 0;
        __syncwarp();
        for (int i = lane; i < n; i += 32)
          if ((rows[i] >> p) & 1u) rows[i] ^= prow;
        if (lane < cnt && ((s_basis[lane] >> p) & 1u)) s_basis[lane] ^= prow;
        __syncwarp();
        if (lane == 0) { s_basis[cnt] = prow; s_piv[cnt] = p; }
        ++cnt;
        __syncwarp();
      }
      if (lane == 0) {
        s_rank = cnt;
        int m = 0, pi = 0;
        for (int j = 0; j < nA; ++j) {
          if (pi < cnt && s_piv[pi] == j) { ++pi; continue; }
          uint32_t mask = 0;
          for (int i = 0; i < cnt; ++i) mask |= ((s_basis[i] >> j) & 1u) << i;
          s_nonpiv[m] = j;
          s_nonpiv_mask[m] = mask;
          ++m;
        }
        s_n_nonpiv = m;
      }
    }
    __syncthreads();

    // --- offset bits (non-pivot A bits) and Z-string values, one warp each ---
    // A non-pivot bit y_j is fixed by the pivot bits: y_j = off_j ^ sum_i
    // B_i[j] y_{piv_i}, so off_j is the sign of <Z_{A_j} prod Z_{A_piv_i}>.
    const int nnp = s_n_nonpiv;
    const int nzu = F.nz << F.qout;
    for (int ev = warp; ev < nnp + nzu; ev += nwarps) {
      uint64_t acc = 0;
      if (ev < nnp) {
        const int j = s_nonpiv[ev];
        const uint32_t mask = s_nonpiv_mask[ev];
        if (lane < W) {
          acc = tab[(size_t)P.wires[F.A_off + j] * W + lane];
          for (int i = 0; i < s_rank; ++i)
            if ((mask >> i) & 1u) acc ^= tab[(size_t)P.wires[F.A_off + s_piv[i]] * W + lane];
        }
        const int z = zexp_from_acc(tab, n, W, Wh, acc, lane, s_sel[warp], R.status);
        if (lane == 0) {
          if (z == 0) atomicOr(R.status, 2u);
          if (z < 0) atomicOr(&s_off, 1u << j);
        }
      } else {
        const int zi = (ev - nnp) >> F.qout, u = (ev - nnp) & ((1 << F.qout) - 1);
        if (lane < W) {
          const int q0 = P.zoffs[F.zw_off + zi], q1 = P.zoffs[F.zw_off + zi + 1];
          for (int q = q0; q < q1; ++q) acc ^= tab[(size_t)P.wires[q] * W + lane];
          for (int o = 0; o < F.qout; ++o)
            if ((u >> o) & 1) acc ^= tab[(size_t)P.wires[F.qout_off + o] * W + lane];
        }
        const int z = zexp_from_acc(tab, n, W, Wh, acc, lane, s_sel[warp], R.status);
        if (lane == 0)
          R.zval[F.zval_off + ((long long)v * F.nz + zi) * (1 << F.qout) + u] = (float)z;
      }
    }
    __syncthreads();
    if (tid == 0) {
      SpaceRec& sp = R.spaces[F.space_off + v];
      sp.off = s_off;
      sp.rank = s_rank;
      for (int i = 0; i < kMaxMeas; ++i) sp.basis[i] = i < s_rank ? s_basis[i] : 0u;
      sp.flags = 0;
    }
    if (E.mode == CCS_EXACT) {
      const int rk = s_rank;
      const float pr = ldexpf(1.0f, -rk);
      float* d = R.dist + F.dist_off + ((long long)v << nA);
      for (int c = tid; c < (1 << rk); c += nt) {
        uint32_t y = s_off;
        for (int i = 0; i < rk; ++i)
          if ((c >> i) & 1) y ^= s_basis[i];
        d[y] = pr;
      }
    }
    __syncthreads();
  }
}

// --- K3: Philox4x32-10 counter-based sampling from the affine space -------
namespace {
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}
}  // namespace

constexpr int kHistSmem = 8192;   // dense per-CTA histogram up to |A| = 13

__global__ void __launch_bounds__(256) sample_kernel(DevPlan P, DevRes R, EvalParams E, int spc,
                                                     int chunks) {
  __shared__ uint32_t tbl[3][256];
  __shared__ uint32_t hist[kHistSmem];
  const int item = blockIdx.x / chunks, chunk = blockIdx.x % chunks;
  const int2 it = P.items_cliff[item];
  const FragDev& F = P.frags[it.x];
  const int v = it.y;
  const SpaceRec& sp = R.spaces[F.space_off + v];
  const int rank = sp.rank, nA = F.nA;
  const uint32_t off = sp.off;
  for (int t = threadIdx.x; t < 3 * 256; t += blockDim.x) {
    const int k = t >> 8, byte = t & 255;
    uint32_t acc = 0;
    for (int b = 0; b < 8; ++b) {
      const int j = 8 * k + b;
      if (j < rank && ((byte >> b) & 1)) acc ^= sp.basis[j];
    }
    tbl[k][byte] = acc;
  }
  const bool smem_hist = (1 << nA) <= kHistSmem;
  if (smem_hist)
    for (int y = threadIdx.x; y < (1 << nA); y += blockDim.x) hist[y] = 0;
  __syncthreads();
  uint32_t* gcounts = R.counts + F.counts_off + ((long long)v << nA);
  const uint32_t cmask = rank >= 32 ? 0xffffffffu : ((1u << rank) - 1u);
  const uint32_t s_end = min((uint32_t)E.shots, (uint32_t)(chunk + 1) * (uint32_t)spc);
  for (uint32_t s = (uint32_t)chunk * spc + threadIdx.x; s < s_end; s += blockDim.x) {
    const uint4 o = philox4x32_10(make_uint4(s, (uint32_t)v, (uint32_t)F.findex, (uint32_t)F.problem),
                                  E.seed_lo, E.seed_hi);
    const uint32_t c = o.x & cmask;
    const uint32_t y = off ^ tbl[0][c & 255] ^ tbl[1][(c >> 8) & 255] ^ tbl[2][(c >> 16) & 255];
    if (smem_hist) atomicAdd(&hist[y], 1u);
    else atomicAdd(&gcounts[y], 1u);
  }
  if (smem_hist) {
    __syncthreads();
    for (int y = threadIdx.x; y < (1 << nA); y += blockDim.x)
      if (hist[y]) atomicAdd(&gcounts[y], hist[y]);
  }
}

cudaError_t launch_clifford(const DevPlan& p, const DevRes& r, const EvalParams& e, int threads,
                            int smem_words, int grid, cudaStream_t s) {
  if (p.n_items_cliff == 0) return cudaSuccess;
  const size_t smem = (size_t)smem_words * 8;
  cudaError_t err = cudaFuncSetAttribute(clifford_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  clifford_kernel<<<grid, threads, smem, s>>>(p, r, e);
  return cudaGetLastError();
}

cudaError_t launch_sample(const DevPlan& p, const DevRes& r, const EvalParams& e, int spc, int threads,
                          cudaStream_t s) {
  if (p.n_items_cliff == 0 || e.shots == 0) return cudaSuccess;
  const int chunks = (int)((e.shots + spc - 1) / spc);
  const long long grid = (long long)p.n_items_cliff * chunks;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  sample_kernel<<<(unsigned)grid, threads, 0, s>>>(p, r, e, spc, chunks);
  return cudaGetLastError();
}

}  // namespace ccs
