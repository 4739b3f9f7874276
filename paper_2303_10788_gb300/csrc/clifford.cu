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
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.cuh"

#include <type_traits>

namespace ccs {

constexpr int kMaxWh = (kMaxBodyQubits + 63) / 64;
constexpr int kZOffStage = 257, kZWireStage = 1024;

namespace {

// 0 or ~0u: bit `bit` of v spread over a word (a constant shift pair once
// `bit` is unrolled).
__device__ __forceinline__ uint32_t bm32(unsigned v, int bit) {
  return (uint32_t)((int32_t)(v << (31 - bit)) >> 31);
}

// Apply one fused Clifford op to this thread's G words wk[0..G) (entries
// >= W are skipped): the op's 31 bit masks are expanded once for all G, as
// 32-bit words, and each 64-row word is updated as two 32-bit halves.
// The words are spread so that one load instruction of a warp touches each
// shared-memory bank pair at most twice (see word_map below).
template <int G>
__device__ __forceinline__ void apply_op_g(CliffordOp op, uint64_t* tab, int W, int zb, const int (&wk)[G],
                                           uint64_t (&rd)[G]) {
  const unsigned M = op.M, A = op.anf;
  uint32_t m[16], a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) { m[i] = bm32(M, i); a[i] = bm32(A, i); }
  uint64_t* pxa = tab + (size_t)op.qa * W;
  uint64_t* pza = tab + (size_t)(zb + op.qa) * W;
  uint64_t* pxb = tab + (size_t)op.qb * W;
  uint64_t* pzb = tab + (size_t)(zb + op.qb) * W;
#pragma unroll
  for (int k = 0; k < G; ++k) {
    const int w = wk[k];
    if (G > 1 && w >= W) continue;
    const uint64_t V0 = pxa[w], V1 = pza[w], V2 = pxb[w], V3 = pzb[w];
    uint32_t r[2], u0[2], u1[2], u2[2], u3[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t v0 = (uint32_t)(V0 >> (32 * h)), v1 = (uint32_t)(V1 >> (32 * h));
      const uint32_t v2 = (uint32_t)(V2 >> (32 * h)), v3 = (uint32_t)(V3 >> (32 * h));
      const uint32_t v01 = v0 & v1, v23 = v2 & v3;
      r[h] = (v0 & a[1]) ^ (v1 & a[2]) ^ (v01 & a[3]) ^ (v2 & a[4]) ^ ((v0 & v2) & a[5]) ^ ((v1 & v2) & a[6]) ^
             ((v01 & v2) & a[7]) ^ (v3 & a[8]) ^ ((v0 & v3) & a[9]) ^ ((v1 & v3) & a[10]) ^
             ((v01 & v3) & a[11]) ^ (v23 & a[12]) ^ ((v0 & v23) & a[13]) ^ ((v1 & v23) & a[14]) ^
             ((v01 & v23) & a[15]);
      u0[h] = (v0 & m[0]) ^ (v1 & m[1]) ^ (v2 & m[2]) ^ (v3 & m[3]);
      u1[h] = (v0 & m[4]) ^ (v1 & m[5]) ^ (v2 & m[6]) ^ (v3 & m[7]);
      u2[h] = (v0 & m[8]) ^ (v1 & m[9]) ^ (v2 & m[10]) ^ (v3 & m[11]);
      u3[h] = (v0 & m[12]) ^ (v1 & m[13]) ^ (v2 & m[14]) ^ (v3 & m[15]);
    }
    rd[k] ^= ((uint64_t)r[1] << 32) | r[0];
    pxa[w] = ((uint64_t)u0[1] << 32) | u0[0];
    pza[w] = ((uint64_t)u1[1] << 32) | u1[0];
    pxb[w] = ((uint64_t)u2[1] << 32) | u2[0];
    pzb[w] = ((uint64_t)u3[1] << 32) | u3[0];
  }
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

// Phase exponent g of the product of two single-qubit Paulis (x1,z1)(x2,z2)
// = i^g (x1^x2, z1^z2), with (1,1) meaning Y (Aaronson-Gottesman, Sec. III).
__device__ __forceinline__ int pauli_g(unsigned x1, unsigned z1, unsigned x2, unsigned z2) {
  if (x1 & z1) return (int)z2 - (int)x2;
  if (x1) return (int)(z2 & 1u) * (2 * (int)x2 - 1);
  if (z1) return (int)x2 * (1 - 2 * (int)z2);
  return 0;
}

// Start a variant from its fragment's body tableau.  The body B is the gate
// sequence U applied to the identity tableau, so its destabilizer row i is
// U X_i U^+ and its stabilizer row i is U Z_i U^+.  Preparing input wire i
// with a one-qubit Clifford C before U turns those rows into
// U (C X_i C^+) U^+ and U (C Z_i C^+) U^+, where C X C^+ and C Z C^+ are
// signed X, Y or Z read off the preparation's fused op (its M columns for x
// and z, its sign polynomial's linear terms).  The image of Y_i = i X_i Z_i
// is i times the product of the two body rows, whose sign follows from the
// summed phase exponents (Sec. III of Aaronson-Gottesman).  Conjugation is
// exact and row-wise, so the result equals simulating C then U bit for bit.
// Phase 1 (one warp per Y-valued input) sums the exponents; phase 2 (one
// thread per column) rewrites the two rows of every input in that column.
__device__ void prep_rows_from_body(const CliffordOp* s_prep, const int* s_qin, const FragDev& F, int v,
                                    uint64_t* tab, int tid, int nt, int* s_code, int* s_ry) {
  const int n = F.n, W = F.W, Wh = F.Wh, zb = n + 1, rcol = 2 * (n + 1), ncol = 2 * n + 3;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  for (int o = tid; o < F.qin; o += nt) {
    const CliffordOp op = s_prep[variant_in_digit(v, o)];
    const unsigned M = op.M, A = op.anf;
    // 2-bit Pauli codes (bit 0 = x, bit 1 = z) and sign bits of the two images
    const int dc = (int)((M >> 0) & 1u) | (int)(((M >> 4) & 1u) << 1);
    const int sc = (int)((M >> 1) & 1u) | (int)(((M >> 5) & 1u) << 1);
    s_code[o] = dc | (sc << 2) | (int)(((A >> 1) & 1u) << 4) | (int)(((A >> 2) & 1u) << 5);
  }
  __syncthreads();
  for (int o = warp; o < F.qin; o += nwarps) {
    const int code = s_code[o];
    if ((code & 3) != 3 && ((code >> 2) & 3) != 3) continue;   // no Y image
    const int i = s_qin[o];
    const int wd = i >> 6, b = i & 63;
    int g = 0;
    for (int j = lane; j < n; j += 32) {
      const unsigned xd = (unsigned)(tab[(size_t)j * W + wd] >> b) & 1u;
      const unsigned zd = (unsigned)(tab[(size_t)(zb + j) * W + wd] >> b) & 1u;
      const unsigned xs = (unsigned)(tab[(size_t)j * W + Wh + wd] >> b) & 1u;
      const unsigned zs = (unsigned)(tab[(size_t)(zb + j) * W + Wh + wd] >> b) & 1u;
      g += pauli_g(xd, zd, xs, zs);
    }
    for (int off = 16; off; off >>= 1) g += __shfl_xor_sync(0xffffffffu, g, off);
    if (lane == 0) {
      const unsigned rd = (unsigned)(tab[(size_t)rcol * W + wd] >> b) & 1u;
      const unsigned rs = (unsigned)(tab[(size_t)rcol * W + Wh + wd] >> b) & 1u;
      const int e = ((1 + g) % 4 + 4) % 4;      // 0 or 2: i D S is Hermitian
      s_ry[o] = (int)(rd ^ rs ^ (e == 2 ? 1u : 0u));
    }
  }
  __syncthreads();
  for (int c = tid; c < ncol; c += nt) {
    uint64_t* col = tab + (size_t)c * W;
    for (int o = 0; o < F.qin; ++o) {
      const int code = s_code[o];
      if (code == (1 | (2 << 2))) continue;      // X -> X, Z -> Z, no signs: unchanged
      const int i = s_qin[o];
      const int wd = i >> 6, b = i & 63;
      const unsigned db = (unsigned)(col[wd] >> b) & 1u, sb = (unsigned)(col[Wh + wd] >> b) & 1u;
      unsigned nd, ns;
      auto img = [&](int pc) -> unsigned {
        if (c == rcol) return pc == 1 ? db : pc == 2 ? sb : (unsigned)s_ry[o];
        return pc == 1 ? db : pc == 2 ? sb : (db ^ sb);
      };
      nd = img(code & 3);
      ns = img((code >> 2) & 3);
      if (c == rcol) {
        nd ^= (unsigned)(code >> 4) & 1u;
        ns ^= (unsigned)(code >> 5) & 1u;
      }
      col[wd] = (col[wd] & ~(1ull << b)) | ((uint64_t)nd << b);
      col[Wh + wd] = (col[Wh + wd] & ~(1ull << b)) | ((uint64_t)ns << b);
    }
  }
  __syncthreads();
}

}  // namespace

namespace {
// Deep, narrow circuits (moments of a few ops: a chain) are bound by the
// latency of each op, not by tableau traffic, so their ops are applied
// cooperatively: eight lanes per op, lane (h, j) producing output column j
// (X_a, Z_a, X_b, Z_b) on 32-bit half h of the word and a quarter of the
// op's sign-flip terms (terms 4j .. 4j+3 of its algebraic normal form, whose
// factors in v2, v3 are fixed by j), reduced over the four lanes of the half
// by shuffles: the arithmetic of apply_op_g, split over lanes.  Every lane of
// the block must call it.
__device__ __forceinline__ void apply_moment_coop(const CliffordOp* ops, int c0, int n_ops, uint32_t* t32, int zb,
                                                  uint64_t& rd) {
  const int lane = threadIdx.x & 31;
  for (int t0 = (int)threadIdx.x - lane; t0 < 8 * n_ops; t0 += (int)blockDim.x) {
    const int t = t0 + lane;
    const bool act = t < 8 * n_ops;
    const int h = (t >> 2) & 1, j = t & 3;
    uint32_t u = 0u, r = 0u, v0 = 0u, v1 = 0u, v2 = 0u, v3 = 0u;
    int col = 0;
    if (act) {
      const CliffordOp op = ops[c0 + (t >> 3)];
      v0 = t32[2 * op.qa + h];
      v1 = t32[2 * (zb + op.qa) + h];
      v2 = t32[2 * op.qb + h];
      v3 = t32[2 * (zb + op.qb) + h];
      const unsigned M = op.M >> (4 * j), A = (op.anf & ~1u) >> (4 * j);   // ANF term 0 is not used
      u = (v0 & bm32(M, 0)) ^ (v1 & bm32(M, 1)) ^ (v2 & bm32(M, 2)) ^ (v3 & bm32(M, 3));
      const uint32_t hi = ((j & 1) ? v2 : ~0u) & ((j & 2) ? v3 : ~0u);
      r = hi & (bm32(A, 0) ^ (v0 & bm32(A, 1)) ^ (v1 & bm32(A, 2)) ^ ((v0 & v1) & bm32(A, 3)));
      col = j == 0 ? op.qa : j == 1 ? zb + op.qa : j == 2 ? op.qb : zb + op.qb;
    }
    r ^= __shfl_xor_sync(0xffffffffu, r, 1);
    r ^= __shfl_xor_sync(0xffffffffu, r, 2);
    __syncwarp();                            // every lane has read its inputs
    if (act) {
      t32[2 * col + h] = u;
      if (j == 0) rd ^= (uint64_t)r << (32 * h);
    }
  }
}
}  // namespace

// --- shared body: one CTA per (Clifford fragment, 64-row word) -------------
// Rows evolve independently under conjugation, so each word of every column
// is an independent problem: the CTA keeps one word per column in shared
// memory and applies the whole op stream to it, moment by moment.
template <bool COOP>   // COOP: eight lanes per op (moments of at most 32 ops)
__global__ void __launch_bounds__(256) body_kernel(DevPlan P, DevRes R, int smem_words) {
  extern __shared__ __align__(16) unsigned long long smem_u64[];
  uint64_t* tab = reinterpret_cast<uint64_t*>(smem_u64);
  const int2 it = P.items_body[blockIdx.x];
  const FragDev& F = P.frags[it.x];
  const int n = F.n, W = F.W, Wh = F.Wh, zb = n + 1, rcol = 2 * (n + 1), ncol = 2 * n + 3;
  const int w = it.y, tid = threadIdx.x, nt = blockDim.x;
  // the op stream and moment offsets follow the column words when they fit
  const int n_ops = P.moments[F.mom_off + F.n_moments];
  const bool staged = ncol + n_ops + (F.n_moments + 2) / 2 + 1 <= smem_words;
  CliffordOp* ops_s = reinterpret_cast<CliffordOp*>(tab + ncol);
  int* mom_s = reinterpret_cast<int*>(tab + ncol + n_ops);
  if (staged) {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(P.cops + F.ops_off);
    for (int i = tid; i < n_ops; i += nt) reinterpret_cast<unsigned long long*>(ops_s)[i] = src[i];
    for (int i = tid; i <= F.n_moments; i += nt) mom_s[i] = P.moments[F.mom_off + i];
  }
  for (int c = tid; c < ncol; c += nt) tab[c] = 0ull;
  __syncthreads();
  {   // identity: destabilizer i = X_i (words [0, Wh)), stabilizer i = Z_i
    const int half = w < Wh ? 0 : 1, i0 = 64 * (w - half * Wh);
    for (int i = i0 + tid; i < min(n, i0 + 64); i += nt) tab[half ? zb + i : i] = 1ull << (i & 63);
  }
  __syncthreads();
  const CliffordOp* ops = staged ? ops_s : P.cops + F.ops_off;
  const int* mom = staged ? mom_s : P.moments + F.mom_off;
  const int wk[1] = {0};
  uint64_t rd[1] = {0ull};
  if (COOP) {
    uint32_t* t32 = reinterpret_cast<uint32_t*>(tab);
    for (int mm = 0; mm < F.n_moments; ++mm) {
      apply_moment_coop(ops, mom[mm], mom[mm + 1] - mom[mm], t32, zb, rd[0]);
      __syncthreads();
    }
  } else if (F.n_moments > 0) {
    // each thread's first op of the next moment is fetched while this
    // moment's op is applied (the op stream does not depend on the tableau)
    int b0 = mom[0], b1 = mom[1];
    CliffordOp nxt{};
    if (b0 + tid < b1) nxt = ops[b0 + tid];
    for (int mm = 0; mm < F.n_moments; ++mm) {
      const int c0 = b0, c1 = b1;
      const CliffordOp cur = nxt;
      if (mm + 1 < F.n_moments) {
        b0 = c1;
        b1 = mom[mm + 2];
        if (b0 + tid < b1) nxt = ops[b0 + tid];
      }
      if (c0 + tid < c1) apply_op_g<1>(cur, tab, 1, zb, wk, rd);
      for (int o = c0 + tid + nt; o < c1; o += nt) apply_op_g<1>(ops[o], tab, 1, zb, wk, rd);
      __syncthreads();
    }
  }
  atomicXor(reinterpret_cast<unsigned long long*>(&tab[rcol]), (unsigned long long)rd[0]);
  __syncthreads();
  unsigned long long* dst = R.body + F.body_off;
  for (int c = tid; c < ncol; c += nt) dst[(size_t)c * W + w] = tab[c];
}

// --- Z images -------------------------------------------------------------
// Pauli expectations of a variant without its tableau.  With the body's rows
// D_j = U X_j U^+ and S_j = U Z_j U^+ (signs included), every Pauli Q on the
// output side decomposes as Q = i^-e (prod_j D_j^a_j)(prod_j S_j^b_j), where
// a_j / b_j say whether Q anticommutes with S_j / D_j (the rows form a
// symplectic basis) and i^e is the phase of that ordered product of rows.
// (D_j commutes with every S_k, k != j, so this order equals the interleaved
// one.)  Conjugating back, U^+ Q U = i^-e X^a Z^b: the backward image.  A
// variant prepares the product state |psi> = (x)_j C_j|0> and measures
// O_o = C'^+ Z C' at quantum output o, so the expectation of a product of
// such Paulis on distinct wires is <psi| prod U^+ Q U |psi>: a product of
// backward images, evaluated on a product state (Aaronson-Gottesman, Sec.
// III, for the row products; the cut identity of Sec. IV for the states and
// observables).  Z-string values and the offsets of rank-deficient outcome
// spaces are both such expectations.
//
// Records of a fragment (2 Wh + 1 words each: a in [0, Wh), b in [Wh, 2Wh),
// the phase exponent -e mod 4 last): k < nz is Z-string k; k = nz + 3 o + d
// is the observable of quantum output o in basis d (0 X, 1 Y, 2 Z: the basis
// changes H, S^+ then H, and none); k = nz + 3 qout + t is Z on marginal
// wire t.
namespace {

__device__ __forceinline__ unsigned long long warp_xor64(unsigned long long x) {
  for (int o = 16; o; o >>= 1) x ^= __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// One record, by one CTA: the anticommutation bits (acc, by warp 0), then
// the ordered row product with its phase, threads over the body's columns.
// The body stays in global memory: a column's W words share one or two
// 128-byte lines, so after the first touch they come from L1.
__device__ void z_image(const DevPlan& P, const DevRes& R, const FragDev& F, int k, unsigned long long* s_sel,
                        unsigned long long* s_ex, unsigned long long* s_ez, int* s_e, unsigned* s_bad) {
  const int n = F.n, W = F.W, Wh = F.Wh, zb = n + 1, rcol = 2 * (n + 1);
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  const unsigned long long* tab = R.body + F.body_off;
  if (tid < Wh) { s_ex[tid] = 0ull; s_ez[tid] = 0ull; }
  if (tid == 0) { *s_e = 0; *s_bad = 0u; }
  __syncthreads();
  if (tid < 32) {
    unsigned long long acc = 0ull;      // lane w < W: anticommutation bits of the rows in word w
    if (k < F.nz) {
      // Z_S: the x-columns of the string's wires, XORed (lanes over wires)
      const int q0 = P.zoffs[F.zw_off + k], q1 = P.zoffs[F.zw_off + k + 1];
      for (int t0 = q0; t0 < q1; t0 += 32) {
        const int wq = t0 + lane < q1 ? P.wires[t0 + lane] : -1;
        if (wq >= 0) atomicXor(&s_ez[wq >> 6], 1ull << (wq & 63));
        for (int w = 0; w < W; ++w) {
          const unsigned long long x = warp_xor64(wq >= 0 ? tab[(size_t)wq * W + w] : 0ull);
          if (lane == w) acc ^= x;
        }
      }
    } else {
      int wq;
      bool ox, oz;
      if (k < F.nz + 3 * F.qout) {
        const int o = (k - F.nz) / 3, d = (k - F.nz) % 3;
        wq = P.wires[F.qout_off + o];
        ox = d != 2;                     // X, Y or Z on wire wq
        oz = d != 0;
      } else {
        wq = P.wires[F.A_off + (k - F.nz - 3 * F.qout)];
        ox = false;
        oz = true;
      }
      if (lane < W) {
        if (ox) acc ^= tab[(size_t)(zb + wq) * W + lane];
        if (oz) acc ^= tab[(size_t)wq * W + lane];
      }
      if (lane == 0) {
        if (ox) s_ex[wq >> 6] = 1ull << (wq & 63);
        if (oz) s_ez[wq >> 6] = 1ull << (wq & 63);
      }
    }
    // destabilizer rows are selected by a (stabilizer-half bits), stabilizer rows by b
    if (lane < W) s_sel[lane < Wh ? lane + Wh : lane - Wh] = acc;
  }
  __syncthreads();
  int e = 0;
  unsigned bad = 0;
  for (int j = tid; j < n; j += nt) {
    unsigned cx = 0, cz = 0;
    const unsigned long long* xc = tab + (size_t)j * W;
    const unsigned long long* zc = tab + (size_t)(zb + j) * W;
    for (int w = 0; w < W; ++w) {
      const unsigned long long sw = s_sel[w];
      const unsigned long long x = xc[w] & sw;
      const unsigned long long z = zc[w] & sw;
      const unsigned long long px = prefix_xor_excl(x) ^ (cx ? ~0ull : 0ull);
      const unsigned long long pz = prefix_xor_excl(z) ^ (cz ? ~0ull : 0ull);
      const unsigned long long X1 = px & ~pz, Y1 = px & pz, Z1 = ~px & pz;
      const unsigned long long X2 = x & ~z, Y2 = x & z, Z2 = ~x & z;
      const unsigned long long plus = (X1 & Y2) | (Y1 & Z2) | (Z1 & X2);
      const unsigned long long minus = (X1 & Z2) | (Y1 & X2) | (Z1 & Y2);
      e += __popcll(plus) - __popcll(minus);
      cx ^= __popcll(x) & 1;
      cz ^= __popcll(z) & 1;
    }
    // the product must be Q itself up to phase
    if (cx != (unsigned)((s_ex[j >> 6] >> (j & 63)) & 1ull) || cz != (unsigned)((s_ez[j >> 6] >> (j & 63)) & 1ull))
      bad = 1;
  }
  if (tid < W) e += 2 * __popcll(tab[(size_t)rcol * W + tid] & s_sel[tid]);
  for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if (lane == 0) atomicAdd(s_e, e);
  if (bad) atomicOr(s_bad, 1u);
  __syncthreads();
  if (tid == 0 && *s_bad) atomicOr(R.status, 1u);
  unsigned long long* out = R.zimg + F.zimg_off + (long long)k * (2 * Wh + 1);
  if (tid < W) out[tid] = s_sel[tid];   // a = sel[0, Wh), b = sel[Wh, 2 Wh)
  if (tid == 0) out[2 * Wh] = (unsigned long long)(((-*s_e) % 4 + 4) % 4);
}

// Expectation in {-1, 0, 1} of a variant (preparation digits `pin`, basis
// digits `pout`, two bits each) for the product of record zi (a Z-string;
// -1 for none) and the measured Paulis M_t, t in `amask` (t < m: Z on
// marginal wire t; t >= m: the observable of output t - m).  The images
// multiply as U^+ Q U = i^E X^A Z^B; then A must vanish off the quantum
// inputs and on input j the pattern (A_j, B_j) must be the prepared state's
// stabilizer (|0>: Z, |1>: -Z, |+>: X, |+i>: Y = i XZ).
__device__ int pauli_value(const unsigned long long* img, const FragDev& F, int zi, uint32_t amask, unsigned pin,
                           unsigned pout, const int* qw, unsigned* status) {
  const int Wh = F.Wh, st = 2 * Wh + 1, m = F.m, zo = F.nz, zm = F.nz + 3 * F.qout;
  auto rec = [&](int t) -> int {
    return t < m ? zm + t : zo + 3 * (t - m) + (int)((pout >> (2 * (t - m))) & 3u);
  };
  int E = zi >= 0 ? (int)img[(size_t)zi * st + 2 * Wh] : 0;
  for (uint32_t h = amask; h; h &= h - 1) E += (int)img[(size_t)rec(__ffs(h) - 1) * st + 2 * Wh];
  for (int w = 0; w < Wh; ++w) {
    unsigned long long A = 0ull, B = 0ull;
    if (zi >= 0) {
      A = img[(size_t)zi * st + w];
      B = img[(size_t)zi * st + Wh + w];
    }
    for (uint32_t h = amask; h; h &= h - 1) {
      const unsigned long long* r = img + (size_t)rec(__ffs(h) - 1) * st;
      const unsigned long long a = r[w];
      E += 2 * __popcll(B & a);
      A ^= a;
      B ^= r[Wh + w];
    }
    for (int i = 0; i < F.qin; ++i) {
      const int q = qw[i];
      if ((q >> 6) != w) continue;
      const unsigned code = (unsigned)((A >> (q & 63)) & 1ull) | ((unsigned)((B >> (q & 63)) & 1ull) << 1);
      A &= ~(1ull << (q & 63));
      if (code == 0) continue;
      const unsigned s = (pin >> (2 * i)) & 3u;       // 0 |0>, 1 |1>, 2 |+>, 3 |+i>
      const unsigned want = s < 2 ? 2u : s == 2 ? 1u : 3u;
      if (code != want) return 0;
      E += s == 1 ? 2 : s == 3 ? 3 : 0;
    }
    if (A) return 0;                                   // X or Y on a |0> input
  }
  E &= 3;
  if (E & 1) {
    atomicOr(status, 1u);
    return 0;
  }
  return E ? -1 : 1;
}

__device__ __forceinline__ unsigned pack_in_digits(int v, int qin) {
  unsigned p = 0;
  for (int i = 0; i < qin; ++i) {
    p |= (unsigned)(v % 4) << (2 * i);
    v /= 4;
  }
  return p;
}
__device__ __forceinline__ unsigned pack_out_digits(int v, int qin, int qout) {
  for (int i = 0; i < qin; ++i) v /= 4;
  unsigned p = 0;
  for (int o = 0; o < qout; ++o) {
    p |= (unsigned)(v % 3) << (2 * o);
    v /= 3;
  }
  return p;
}

// Fold the lanes' rows (bits < nA) into a warp's echelon basis: lane p holds
// the vector with pivot p in `mine`, `have` the pivot set (warp-uniform).
__device__ __forceinline__ void absorb32(uint32_t row, uint32_t& have, uint32_t& mine, int nA, int lane) {
  const unsigned FULLW = 0xffffffffu;
  for (uint32_t h = have; h; h &= h - 1) {
    const int p = __ffs(h) - 1;
    const uint32_t bp = __shfl_sync(FULLW, mine, p);
    if ((row >> p) & 1u) row ^= bp;
  }
  for (int p = 0; p < nA; ++p) {
    if ((have >> p) & 1u) continue;
    const unsigned msk = __ballot_sync(FULLW, (row >> p) & 1u);
    if (!msk) continue;
    const int leader = __ffs(msk) - 1;
    const uint32_t prow = __shfl_sync(FULLW, row, leader);
    if (lane == leader) row = 0;
    else if ((row >> p) & 1u) row ^= prow;
    if (lane == p) mine = prow;
    have |= 1u << p;
  }
}

// Projection of an extended vector (X bits on A, then Z bits on the quantum
// outputs) through output basis digits pout (0 X, 1 Y, 2 Z): the X bit of
// output o becomes its observable's anticommutation bit, z for X, x ^ z for
// Y, x for Z.
__device__ __forceinline__ uint32_t project_ext(unsigned long long e, int nA, int m, int qout, unsigned pout) {
  uint32_t keepX = (1u << m) - 1u, fromZ = 0u;
  for (int o = 0; o < qout; ++o) {
    const unsigned d = (pout >> (2 * o)) & 3u;
    if (d != 0) keepX |= 1u << (m + o);
    if (d != 2) fromZ |= 1u << (m + o);
  }
  const uint32_t x = (uint32_t)(e & ((1ull << nA) - 1ull));
  const uint32_t z = (uint32_t)((e >> nA) << m);
  return (x & keepX) ^ (z & fromZ);
}

// Fold `row` into the warp's echelon basis eb[] (pivot slots) / have.
__device__ __forceinline__ void absorb64(unsigned long long row, unsigned long long* eb, unsigned long long& have,
                                         int ne, int lane) {
  for (unsigned long long h = have; h; h &= h - 1) {
    const int p = __ffsll((long long)h) - 1;
    if ((row >> p) & 1ull) row ^= eb[p];
  }
  for (int p = 0; p < ne; ++p) {
    if ((have >> p) & 1ull) continue;
    const unsigned msk = __ballot_sync(0xffffffffu, (unsigned)((row >> p) & 1ull));
    if (!msk) continue;
    const int leader = __ffs(msk) - 1;
    const unsigned long long prow = __shfl_sync(0xffffffffu, row, leader);
    if (lane == leader) row = 0ull;
    else if ((row >> p) & 1ull) row ^= prow;
    if (lane == 0) eb[p] = prow;
    have |= 1ull << p;
    __syncwarp();
  }
}
}  // namespace

// --- shared-row basis, Z images and offset table ----------------------------
// CTAs [0, n_cliff_frags): one per Clifford fragment.  Every variant keeps
// the body's stabilizer rows outside its quantum inputs; only the input rows
// and the output columns change.  The rank of a variant's measured set A
// therefore follows from the span of those shared rows, taken as extended
// vectors e_i = (X bits on A, Z bits on the quantum outputs) so that any
// output basis change maps them linearly.  The CTA stores an echelon basis
// of that span (pivot = lowest set bit) in 64 pivot slots plus the pivot mask.
// CTAs after those: one Z-image record each.  The last CTA to finish a
// fragment's measurement records (Z of every marginal wire, X / Y / Z of
// every quantum output: counted in R.fragcnt) writes the fragment's offset
// table for rank-deficient variants: record r (r < m: marginal wire r;
// r = m + 3 o + d: output o in basis d) gets its phase, its (a, b) bits on
// the quantum inputs, and the parities popc(b_k & a_r) mod 2 for every
// record k, so that the phase of any product of records needs no vectors.
__global__ void __launch_bounds__(256) body_basis_kernel(DevPlan P, DevRes R) {
  __shared__ unsigned long long s_eb[8][64];
  __shared__ unsigned long long s_eh[8];
  __shared__ int s_col[64];
  __shared__ int s_in[kMaxCuts];
  __shared__ unsigned long long s_cw[64][kMaxWh];   // stabilizer halves of the extended columns
  __shared__ unsigned long long s_zs[4 * kMaxWh];   // record scratch: sel (2 Wh), expected x, expected z
  __shared__ int s_e;
  __shared__ unsigned s_bad, s_last;
  __shared__ unsigned long long s_ct[64];
  __shared__ unsigned long long s_qd[kMaxCuts], s_qs[kMaxCuts];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  if ((int)blockIdx.x >= P.n_cliff_frags) {
    const int2 it = P.items_zimg[(int)blockIdx.x - P.n_cliff_frags];   // (fragment, record)
    const FragDev& F = P.frags[it.x];
    z_image(P, R, F, it.y, s_zs, s_zs + 2 * kMaxWh, s_zs + 3 * kMaxWh, &s_e, &s_bad);
    if (it.y < F.nz) return;                       // string records take no part in the table
    const int m = F.m, Wh = F.Wh, nrec = m + 3 * F.qout, zm = F.nz + 3 * F.qout, st = 2 * Wh + 1;
    const int fi = (int)(F.rb_off / kRowBasisWords);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&R.fragcnt[fi], 1u) == (unsigned)(nrec - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid < 64) s_ct[tid] = 0ull;
    if (tid < F.qin) s_in[tid] = P.wires[F.qin_off + tid];
    __syncthreads();
    const unsigned long long* img = R.zimg + F.zimg_off;
    auto recp = [&](int r) { return img + (size_t)(r < m ? zm + r : F.nz + (r - m)) * st; };
    for (int pr = tid; pr < nrec * nrec; pr += nt) {
      const int l = pr / nrec, k = pr % nrec;       // bit k of ct[l]: popc(b_k & a_l) mod 2
      const unsigned long long* ak = recp(k);
      const unsigned long long* al = recp(l);
      int c = 0;
      for (int w = 0; w < Wh; ++w) c += __popcll(__ldcg(ak + Wh + w) & __ldcg(al + w));
      if (c & 1) atomicOr(&s_ct[l], 1ull << k);
    }
    __syncthreads();
    unsigned long long* out = R.rowbasis + F.rb_off;
    for (int r = tid; r < 64; r += nt) {
      unsigned long long info = 0ull;
      if (r < nrec) {
        const unsigned long long* ar = recp(r);
        info = __ldcg(ar + 2 * Wh) & 3ull;
        for (int i = 0; i < F.qin; ++i) {
          const int q = s_in[i];
          info |= ((__ldcg(ar + (q >> 6)) >> (q & 63)) & 1ull) << (2 + i);
          info |= ((__ldcg(ar + Wh + (q >> 6)) >> (q & 63)) & 1ull) << (16 + i);
        }
      }
      out[65 + r] = r < nrec ? s_ct[r] : 0ull;
      out[129 + r] = info;
    }
    return;
  }
  const FragDev& F = P.frags[P.cliff_frags[blockIdx.x]];
  const int n = F.n, W = F.W, Wh = F.Wh, zb = n + 1, nA = F.nA, ne = F.nA + F.qout;
  for (int j = tid; j < ne; j += nt) s_col[j] = j < nA ? P.wires[F.A_off + j] : zb + P.wires[F.qout_off + j - nA];
  if (tid < F.qin) {
    s_in[tid] = P.wires[F.qin_off + tid];
    s_qd[tid] = 0ull;
    s_qs[tid] = 0ull;
  }
  __syncthreads();
  const unsigned long long* body = R.body + F.body_off;
  for (int t = tid; t < ne * Wh; t += nt) s_cw[t / Wh][t % Wh] = body[(size_t)s_col[t / Wh] * W + Wh + t % Wh];
  // each quantum input's destabilizer and stabilizer rows as extended vectors
  for (int t = tid; t < F.qin * ne; t += nt) {
    const int i = t / ne, j = t % ne, q = s_in[i];
    const unsigned long long* col = body + (size_t)s_col[j] * W;
    if ((col[q >> 6] >> (q & 63)) & 1ull) atomicOr(&s_qd[i], 1ull << j);
    if ((col[Wh + (q >> 6)] >> (q & 63)) & 1ull) atomicOr(&s_qs[i], 1ull << j);
  }
  __syncthreads();
  if (tid < F.qin) {
    R.rowbasis[F.rb_off + kRbInputRows + tid] = s_qd[tid];
    R.rowbasis[F.rb_off + kRbInputRows + kMaxCuts + tid] = s_qs[tid];
  }
  unsigned long long have = 0ull;
  for (int i0 = warp * 32; i0 < n; i0 += nt) {
    const int i = i0 + lane;
    bool shared_row = i < n;
    for (int k = 0; k < F.qin; ++k) shared_row = shared_row && s_in[k] != i;
    unsigned long long row = 0ull;
    if (shared_row) {
      const int w = i >> 6, b = i & 63;
      for (int j = 0; j < ne; ++j) row |= ((s_cw[j][w] >> b) & 1ull) << j;
    }
    absorb64(row, s_eb[warp], have, ne, lane);
  }
  for (int stride = 1; stride < nwarps; stride <<= 1) {
    const bool top = (warp % (2 * stride)) == 0 && warp + stride < nwarps;
    const bool give = (warp % (2 * stride)) == stride;
    if (give && lane == 0) s_eh[warp] = have;
    __syncthreads();
    if (top) {
      const int pw = warp + stride;
      const unsigned long long ph = s_eh[pw];
      absorb64(((ph >> lane) & 1ull) ? s_eb[pw][lane] : 0ull, s_eb[warp], have, ne, lane);
      absorb64(((ph >> (lane + 32)) & 1ull) ? s_eb[pw][lane + 32] : 0ull, s_eb[warp], have, ne, lane);
    }
    __syncthreads();
  }
  if (warp == 0) {
    unsigned long long* out = R.rowbasis + F.rb_off;
    for (int p = lane; p < 64; p += 32) out[p] = ((have >> p) & 1ull) ? s_eb[0][p] : 0ull;
    if (lane == 0) {
      out[64] = have;
      s_eh[0] = have;
    }
  }
}

// The shared rows' basis projected through one output basis combination of
// one fragment (one warp per (fragment, combination); the screen reads the
// result instead of projecting per variant).
__global__ void __launch_bounds__(256) proj_kernel(DevPlan P, DevRes R) {
  const int lane = threadIdx.x & 31;
  const int item = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (item >= P.n_items_proj) return;
  const int2 it = P.items_proj[item];
  const FragDev& F = P.frags[it.x];
  const int pc = it.y, nA = F.nA;
  const unsigned long long* rb = R.rowbasis + F.rb_off;
  const unsigned long long sh = rb[64];
  unsigned pout = 0;
  for (int o = 0, t = pc; o < F.qout; ++o, t /= 3) pout |= (unsigned)(t % 3) << (2 * o);
  uint32_t h32 = 0, mine = 0;
  absorb32(((sh >> lane) & 1ull) ? project_ext(rb[lane], nA, F.m, F.qout, pout) : 0u, h32, mine, nA, lane);
  absorb32(((sh >> (lane + 32)) & 1ull) ? project_ext(rb[lane + 32], nA, F.m, F.qout, pout) : 0u, h32, mine, nA,
           lane);
  uint32_t* pb = R.pbasis + F.pb_off + 25ll * pc;
  if (lane < 24) pb[lane] = ((h32 >> lane) & 1u) ? mine : 0u;
  if (lane == 0) pb[24] = h32;
}

// --- screen -----------------------------------------------------------------
// CTAs [0, rank_blocks): one warp per Clifford variant.  The variant's rows
// on A are the shared rows mapped through its output basis changes (the X
// bit of output o becomes its observable's anticommutation bit: z for X,
// x ^ z for Y, x for Z) plus its new input rows (the image of C Z_i C^+
// under the body: D_i, S_i or their product, bits only).  Ballot
// elimination of those vectors gives the echelon basis of the variant's
// outcome space, back-substitution its unique reduced form.  Each non-pivot
// bit j is fixed by the pivot bits, y_j = off_j ^ sum_i B_i[j] y_piv_i, so
// off_j is the sign of <M_j prod_i M_piv_i> (B_i[j] set), from the Z images
// (every bit is 0 at full rank).  No tableau is formed; the tableau kernel
// runs instead of the screen only when tableaus are kept.
// CTAs after those: (fragment, first variant) blocks of Z-string values:
// the fragment's records staged in shared memory (img_words of them at
// most), one (variant, string) pair per thread, every output subset u.
__global__ void __launch_bounds__(256) screen_kernel(DevPlan P, DevRes R, EvalParams E, int rank_blocks,
                                                     int img_words) {
  extern __shared__ __align__(16) unsigned long long s_img[];
  __shared__ int s_qw[kMaxCuts];
  const int lane = threadIdx.x & 31;
  const unsigned FULLW = 0xffffffffu;
  if ((int)blockIdx.x >= rank_blocks) {
    const int2 zbk = P.zblocks[(int)blockIdx.x - rank_blocks];
    const FragDev& F = P.frags[zbk.x];
    const int nz = F.nz, qout = F.qout, vpb = zblock_variants(nz);
    const int v0 = zbk.y, vcnt = min(vpb, F.nv - v0);
    const int words = (nz + 3 * qout + F.m) * (2 * F.Wh + 1);
    const unsigned long long* img = R.zimg + F.zimg_off;
    if (words <= img_words) {
      for (int i = threadIdx.x; i < words; i += blockDim.x) s_img[i] = img[i];
      img = s_img;
    }
    if (threadIdx.x < F.qin) s_qw[threadIdx.x] = P.wires[F.qin_off + threadIdx.x];
    __syncthreads();
    const int nq = 1 << qout;
    for (int idx = threadIdx.x; idx < vcnt * nz; idx += blockDim.x) {
      const int v = v0 + idx / nz, zi = idx % nz;
      const unsigned pin = pack_in_digits(v, F.qin), pout = pack_out_digits(v, F.qin, qout);
      float* zv = R.zval + F.zval_off + ((long long)v * nz + zi) * nq;
      for (int u = 0; u < nq; ++u)
        zv[u] = (float)pauli_value(img, F, zi, (uint32_t)u << F.m, pin, pout, s_qw, R.status);
    }
    return;
  }
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int tw = (rank_blocks * blockDim.x) >> 5;
  for (int item = gw; item < P.n_items_cliff; item += tw) {
    const int2 it = P.items_cliff[item];
    const FragDev& F = P.frags[it.x];
    const int v = it.y;
    const int nA = F.nA, m = F.m, qout = F.qout;
    const unsigned pin = pack_in_digits(v, F.qin), pout = pack_out_digits(v, F.qin, qout);
    // output basis maps: keepX / fromZ masks over A bits m..m+qout-1
    uint32_t keepX = (1u << m) - 1u, fromZ = 0u;
    for (int o = 0; o < qout; ++o) {
      const unsigned d = (pout >> (2 * o)) & 3u;     // 0 X, 1 Y, 2 Z
      if (d != 0) keepX |= 1u << (m + o);
      if (d != 2) fromZ |= 1u << (m + o);
    }
    auto project = [&](unsigned long long e) -> uint32_t {
      const uint32_t x = (uint32_t)(e & ((1ull << nA) - 1ull));
      const uint32_t z = (uint32_t)((e >> nA) << m);
      return (x & keepX) ^ (z & fromZ);
    };
    uint32_t have = 0, mine = 0;
    auto absorb = [&](uint32_t row) { absorb32(row, have, mine, nA, lane); };
    const unsigned long long* rb = R.rowbasis + F.rb_off;
    if (F.pb_off >= 0) {   // the shared rows' basis for this output basis combination
      int pc = v;
      for (int i = 0; i < F.qin; ++i) pc >>= 2;
      const uint32_t* pb = R.pbasis + F.pb_off + 25ll * pc;
      have = pb[24];
      mine = lane < 24 ? pb[lane] : 0u;
    } else {
      const unsigned long long sh = rb[64];
      absorb(((sh >> lane) & 1ull) ? project(rb[lane]) : 0u);
      absorb(((sh >> (lane + 32)) & 1ull) ? project(rb[lane + 32]) : 0u);
    }
    {   // new stabilizer rows of the quantum inputs (bits only): the image of
        // C Z C^+ is D, S or their product, from the fragment's input rows
      uint32_t row = 0;
      if (lane < F.qin) {
        const unsigned s = (pin >> (2 * lane)) & 3u;
        const int sc = s < 2 ? 2 : s == 2 ? 1 : 3;   // image of Z under the preparation: 1 X, 2 Z, 3 Y
        const unsigned long long e = ((sc & 1) ? rb[kRbInputRows + lane] : 0ull) ^
                                     ((sc & 2) ? rb[kRbInputRows + kMaxCuts + lane] : 0ull);
        row = project(e);
      }
      absorb(row);
    }
    // reduced form in pivot order; non-pivot bits' relations by ballot
    uint32_t vec = ((have >> lane) & 1u) ? mine : 0u;
    for (int q = nA - 1; q > 0; --q) {
      if (!((have >> q) & 1u)) continue;
      const uint32_t bq = __shfl_sync(FULLW, vec, q);
      if (lane < q && ((vec >> q) & 1u)) vec ^= bq;
    }
    const int rank = __popc(have);
    uint32_t off = 0;
    if (rank < nA) {
      uint32_t amask = 0;
      for (int j = 0; j < nA; ++j) {
        if ((have >> j) & 1u) continue;
        const unsigned bm = __ballot_sync(FULLW, ((have >> lane) & 1u) && ((vec >> j) & 1u));
        if (lane == j) amask = bm | (1u << j);
      }
      // sign of <M_j prod M_piv> from the offset table: phases, pairwise
      // commutation parities (product in ascending t) and the prepared inputs
      int E = 0;
      unsigned qa = 0, qb = 0;
      unsigned long long S = 0ull;
      for (uint32_t h = amask; h; h &= h - 1) {
        const int t = __ffs(h) - 1;
        const int r = t < m ? t : m + 3 * (t - m) + (int)((pout >> (2 * (t - m))) & 3u);
        const unsigned long long ct = rb[65 + r], info = rb[129 + r];
        E += (int)(info & 3ull) + 2 * (__popcll(ct & S) & 1);
        S |= 1ull << r;
        qa ^= (unsigned)(info >> 2) & 0x3fffu;
        qb ^= (unsigned)(info >> 16) & 0x3fffu;
      }
      bool bad = false;
      for (int i = 0; i < F.qin; ++i) {
        const unsigned code = ((qa >> i) & 1u) | (((qb >> i) & 1u) << 1);
        if (!code) continue;
        const unsigned s = (pin >> (2 * i)) & 3u;       // 0 |0>, 1 |1>, 2 |+>, 3 |+i>
        bad = bad || code != (s < 2 ? 2u : s == 2 ? 1u : 3u);
        E += s == 1 ? 2 : s == 3 ? 3 : 0;
      }
      if (amask && (bad || (E & 1))) atomicOr(R.status, 2u);
      off = __ballot_sync(FULLW, amask != 0 && (E & 2) != 0);
    }
    SpaceRec& sp = R.spaces[F.space_off + v];
    if ((have >> lane) & 1u) sp.basis[__popc(have & ((1u << lane) - 1u))] = vec;
    else if (lane >= rank && lane < kMaxMeas) sp.basis[lane] = 0u;
    if (lane == 0) {
      sp.off = off;
      sp.rank = rank;
      sp.flags = 0u;
    }
    __syncwarp();
    if (E.mode == CCS_EXACT || (E.mode == CCS_STITCH && F.role != 1)) {
      const float pr = ldexpf(1.0f, -rank);
      float* d = R.dist + F.dist_off + ((long long)v << nA);
      if (rank == nA) {
        for (int y = lane; y < (1 << nA); y += 32) d[y] = pr;
      } else {
        for (int c = lane; c < (1 << rank); c += 32) {   // off ^ the basis vectors c selects
          uint32_t y = off;
          for (int i = 0; i < rank; ++i)
            if ((c >> i) & 1) y ^= sp.basis[i];
          d[y] = pr;
        }
      }
    }
  }
}

// G = words of one op per thread (the op's masks are expanded once per G).
template <int G>
__global__ void __launch_bounds__(512) clifford_kernel(DevPlan P, DevRes R, EvalParams E, int smem_words) {
  extern __shared__ __align__(16) unsigned long long smem_u64[];
  uint64_t* tab = reinterpret_cast<uint64_t*>(smem_u64);
  __shared__ FragDev sF;
  __shared__ int s_item;
  __shared__ int s_rank;
  __shared__ uint32_t s_off;
  __shared__ uint32_t s_basis[kMaxMeas];
  __shared__ int s_piv[kMaxMeas];
  __shared__ uint32_t s_nonpiv_mask[kMaxMeas];   // pivots whose basis row has bit j
  __shared__ int s_nonpiv[kMaxMeas];
  __shared__ int s_n_nonpiv;
  __shared__ uint64_t s_sel[16][kMaxWh];
  __shared__ int s_code[kMaxCuts], s_ry[kMaxCuts];
  __shared__ int s_A[kMaxMeas];                  // local wires of the measured set A
  __shared__ int s_zo[kZOffStage], s_zw[kZWireStage];   // Z-string wire lists (staged when they fit)
  __shared__ bool s_zstaged;
  __shared__ int s_qin[kMaxCuts], s_qout[kMaxCuts];   // local wires of the quantum inputs / outputs
  __shared__ CliffordOp s_prep[4], s_bops[3];    // preparation and basis-change ops
  __shared__ uint32_t s_wb[16][32];              // K2: a warp's basis vectors by pivot
  __shared__ uint32_t s_wh[16];                  // K2: that warp's pivot set

  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  if (tid < 4) s_prep[tid] = P.prep_ops[tid];
  else if (tid < 7) s_bops[tid - 4] = P.basis_ops[tid - 4];   // ordered by the loop's first barrier

  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(&R.work[0], 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= P.n_items_cliff) break;
    const int2 it = P.items_cliff[item];
    {   // the fragment record, once per item, into shared memory
      const int* src = reinterpret_cast<const int*>(P.frags + it.x);
      int* dst = reinterpret_cast<int*>(&sF);
      for (int i = tid; i < (int)(sizeof(FragDev) / 4); i += nt) dst[i] = src[i];
    }
    __syncthreads();
    const FragDev& F = sF;
    const int v = it.y;
    for (int j = tid; j < F.nA; j += nt) s_A[j] = P.wires[F.A_off + j];   // ordered by the next barrier
    if (tid < F.qin) s_qin[tid] = P.wires[F.qin_off + tid];
    else if (tid >= 32 && tid - 32 < F.qout) s_qout[tid - 32] = P.wires[F.qout_off + tid - 32];
    if (F.nz > 0) {   // Z-string wire lists, when they fit
      const int zb0 = P.zoffs[F.zw_off], ztot = P.zoffs[F.zw_off + F.nz] - zb0;
      const bool fit = F.nz + 1 <= kZOffStage && ztot <= kZWireStage;
      if (tid == 0) s_zstaged = fit;
      if (fit) {
        for (int k = tid; k <= F.nz; k += nt) s_zo[k] = P.zoffs[F.zw_off + k] - zb0;
        for (int t = tid; t < ztot; t += nt) s_zw[t] = P.wires[zb0 + t];
      }
    }
    const int n = F.n, W = F.W, Wh = F.Wh, zb = n + 1, rcol = 2 * (n + 1);
    const int ncol = 2 * n + 3;
    // Word map: an op is applied by ngrp = ceil(W/G) threads; thread g of op
    // slot j owns words g + ngrp*((k + j) mod G), k < G.  For a fixed k the
    // slots of a warp cycle through the G blocks of ngrp words, so when W is
    // a multiple of 16 (every column starts at bank pair 0) each 64-bit bank
    // pair sees exactly two accesses per load: conflict-free.
    const int ngrp = (W + G - 1) / G;
    const int J = nt / ngrp;                 // op slots
    const int gidx = tid % ngrp, jslot = tid / ngrp;
    const bool active = jslot < J;
    int wk[G];
#pragma unroll
    for (int k = 0; k < G; ++k) wk[k] = gidx + ngrp * ((k + jslot) % G);
    uint64_t rd[G];
#pragma unroll
    for (int k = 0; k < G; ++k) rd[k] = 0;
    if (E.shared_body) {
      // --- K1 from the fragment's shared body: copy it, rewrite the input rows ---
      const ulonglong2* src = reinterpret_cast<const ulonglong2*>(R.body + F.body_off);
      ulonglong2* dst2 = reinterpret_cast<ulonglong2*>(tab);
      for (int i = tid; i < ncol * W / 2; i += nt) dst2[i] = src[i];
      __syncthreads();
      prep_rows_from_body(s_prep, s_qin, F, v, tab, tid, nt, s_code, s_ry);
    } else {
      // op stream and moment offsets staged after the tableau when they fit
      const int base_words = ncol * W + (n + 1) / 2 + 2;
      const int n_ops = P.moments[F.mom_off + F.n_moments];
      const bool staged = base_words + n_ops + (F.n_moments + 2) / 2 + 2 <= smem_words;
      CliffordOp* ops_s = reinterpret_cast<CliffordOp*>(tab + base_words);
      int* mom_s = reinterpret_cast<int*>(tab + base_words + n_ops);
      const CliffordOp* ops = staged ? ops_s : P.cops + F.ops_off;
      const int* mom = staged ? mom_s : P.moments + F.mom_off;
      if (staged) {
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(P.cops + F.ops_off);
        for (int i = tid; i < n_ops; i += nt) reinterpret_cast<unsigned long long*>(ops_s)[i] = src[i];
        for (int i = tid; i <= F.n_moments; i += nt) mom_s[i] = P.moments[F.mom_off + i];
      }

      // --- K1: initial tableau (destabilizer i = X_i, stabilizer i = Z_i) ---
      for (int i = tid; i < ncol * W; i += nt) tab[i] = 0ull;
      __syncthreads();
      for (int j = tid; j < n; j += nt) {
        tab[(size_t)j * W + (j >> 6)] = 1ull << (j & 63);
        tab[(size_t)(zb + j) * W + Wh + (j >> 6)] = 1ull << (j & 63);
      }
      __syncthreads();

      if (active) {                          // preparations at quantum inputs
        for (int o = jslot; o < F.qin; o += J) {
          CliffordOp op = s_prep[variant_in_digit(v, o)];
          op.qa = (uint16_t)s_qin[o];
          op.qb = (uint16_t)n;
          apply_op_g<G>(op, tab, W, zb, wk, rd);
        }
      }
      __syncthreads();
      for (int mm = 0; mm < F.n_moments; ++mm) {
        const int b0 = mom[mm], b1 = mom[mm + 1];
        if (active)
          for (int o = b0 + jslot; o < b1; o += J) apply_op_g<G>(ops[o], tab, W, zb, wk, rd);
        __syncthreads();
      }
    }
    if (active) {                          // basis changes at quantum outputs
      for (int o = jslot; o < F.qout; o += J) {
        CliffordOp op = s_bops[variant_out_digit(v, F.qin, o)];
        op.qa = (uint16_t)s_qout[o];
        op.qb = (uint16_t)n;
        apply_op_g<G>(op, tab, W, zb, wk, rd);
      }
#pragma unroll
      for (int k = 0; k < G; ++k)
        if (wk[k] < W)
          atomicXor(reinterpret_cast<unsigned long long*>(&tab[(size_t)rcol * W + wk[k]]),
                    (unsigned long long)rd[k]);
    }
    __syncthreads();

    if (E.keep_tableaus && F.tab_off >= 0) {
      unsigned long long* dst = R.tabs + F.tab_off + (long long)v * ncol * W;
      for (int i = tid; i < ncol * W; i += nt) dst[i] = tab[i];
    }

    // --- K2: basis B = RREF of the stabilizer X-block on the columns A ---
    // Every warp takes its stabilizer rows (lane = row, bits = A columns) and
    // builds an echelon basis of them with ballots (pivot = lowest set bit,
    // lane p keeps the vector with pivot p).  The warp bases are merged in a
    // binary tree (the partner's vectors are reduced by the own pivots, then
    // eliminated among themselves), and warp 0 back-substitutes the final
    // basis into the unique reduced form, in pivot order.
    const int nA = F.nA;
    if (tid == 0) s_off = 0;
    const unsigned FULLW = 0xffffffffu;
    uint32_t mine = 0, have = 0;
    auto absorb = [&](uint32_t row) {
      for (uint32_t h = have; h; h &= h - 1) {
        const int p = __ffs(h) - 1;
        const uint32_t bp = __shfl_sync(FULLW, mine, p);
        if ((row >> p) & 1u) row ^= bp;
      }
      for (int p = 0; p < nA; ++p) {
        if ((have >> p) & 1u) continue;
        const unsigned msk = __ballot_sync(FULLW, (row >> p) & 1u);
        if (!msk) continue;
        const int leader = __ffs(msk) - 1;
        const uint32_t prow = __shfl_sync(FULLW, row, leader);
        if (lane == leader) row = 0;
        else if ((row >> p) & 1u) row ^= prow;
        if (lane == p) mine = prow;
        have |= 1u << p;
      }
    };
    for (int i0 = warp * 32; i0 < n; i0 += nt) {
      const int i = i0 + lane;
      uint32_t row = 0;
      if (i < n) {
        const size_t w = (size_t)Wh + (i >> 6);
        const int b = i & 63;
        for (int j = 0; j < nA; ++j) row |= (uint32_t)((tab[(size_t)s_A[j] * W + w] >> b) & 1ull) << j;
      }
      absorb(row);
    }
    for (int stride = 1; stride < nwarps; stride <<= 1) {
      const bool top = (warp % (2 * stride)) == 0 && warp + stride < nwarps;
      const bool give = (warp % (2 * stride)) == stride;
      if (give) {
        s_wb[warp][lane] = mine;
        if (lane == 0) s_wh[warp] = have;
      }
      __syncthreads();
      if (top) {
        const int pw = warp + stride;
        absorb(((s_wh[pw] >> lane) & 1u) ? s_wb[pw][lane] : 0u);
      }
      __syncthreads();
    }
    if (warp == 0) {
      uint32_t vec = ((have >> lane) & 1u) ? mine : 0u;
      for (int q = nA - 1; q > 0; --q) {
        if (!((have >> q) & 1u)) continue;
        const uint32_t bq = __shfl_sync(FULLW, vec, q);
        if (lane < q && ((vec >> q) & 1u)) vec ^= bq;
      }
      const int cnt = __popc(have);
      if (lane < nA && ((have >> lane) & 1u)) {
        const int pos = __popc(have & ((1u << lane) - 1u));
        s_basis[pos] = vec;
        s_piv[pos] = lane;
      }
      __syncwarp();
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
    const int nzs = F.nz;
    for (int ev = warp; ev < nnp + nzs; ev += nwarps) {
      if (ev < nnp) {
        uint64_t acc = 0;
        const int j = s_nonpiv[ev];
        const uint32_t mask = s_nonpiv_mask[ev];
        if (lane < W) {
          acc = tab[(size_t)s_A[j] * W + lane];
          for (int i = 0; i < s_rank; ++i)
            if ((mask >> i) & 1u) acc ^= tab[(size_t)s_A[s_piv[i]] * W + lane];
        }
        const int z = zexp_from_acc(tab, n, W, Wh, acc, lane, s_sel[warp], R.status);
        if (lane == 0) {
          if (z == 0) atomicOr(R.status, 2u);
          if (z < 0) atomicOr(&s_off, 1u << j);
        }
      } else {
        // Z-string zi: its own columns once, then every subset u of the outputs
        const int zi = ev - nnp;
        uint64_t acc0 = 0;
        if (lane < W) {
          if (s_zstaged) {
            for (int q = s_zo[zi]; q < s_zo[zi + 1]; ++q) acc0 ^= tab[(size_t)s_zw[q] * W + lane];
          } else {
            const int q0 = P.zoffs[F.zw_off + zi], q1 = P.zoffs[F.zw_off + zi + 1];
            for (int q = q0; q < q1; ++q) acc0 ^= tab[(size_t)P.wires[q] * W + lane];
          }
        }
        for (int u = 0; u < (1 << F.qout); ++u) {
          uint64_t acc = acc0;
          if (lane < W)
            for (int o = 0; o < F.qout; ++o)
              if ((u >> o) & 1) acc ^= tab[(size_t)s_qout[o] * W + lane];
          const int z = zexp_from_acc(tab, n, W, Wh, acc, lane, s_sel[warp], R.status);
          if (lane == 0) R.zval[F.zval_off + ((long long)v * F.nz + zi) * (1 << F.qout) + u] = (float)z;
        }
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
    if (E.mode == CCS_EXACT || (E.mode == CCS_STITCH && F.role != 1)) {
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

// Lookup tables of a variant's affine space: tbl[k][byte] = XOR of the basis
// vectors 8k + b selected by byte's bits, only for the ceil(rank / 8)
// groups that exist (entry 0 of the others is 0, which is all a shot of
// rank-limited coefficients can select there).  The basis is read once into
// shared memory; every thread of the block must call this (it synchronises).
__device__ __forceinline__ void build_tables(uint32_t (*tbl)[256], const SpaceRec& sp, int rank) {
  __shared__ uint32_t s_b[kMaxMeas];
  const int ntab = rank > 16 ? 3 : rank > 8 ? 2 : 1;
  if ((int)threadIdx.x < kMaxMeas) s_b[threadIdx.x] = (int)threadIdx.x < rank ? sp.basis[threadIdx.x] : 0u;
  __syncthreads();
  for (int t = threadIdx.x; t < ntab * 256; t += blockDim.x) {
    const int k = t >> 8, byte = t & 255;
    uint32_t acc = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
      if ((byte >> b) & 1) acc ^= s_b[8 * k + b];
    tbl[k][byte] = acc;
  }
  if ((int)threadIdx.x < 3 - ntab) tbl[ntab + threadIdx.x][0] = 0u;
}

// --- K3: Philox4x32-10 counter-based sampling from the affine space -------
namespace {
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // each 32 x 32 -> 64-bit product is one wide multiply (high and low words);
    // the round keys are launch constants
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.k[r][0], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ K.k[r][1],
                   (uint32_t)p0);
  }
  return c;
}
// Shots [t0, t1) of one variant (t0 a multiple of 4 x fields per word),
// threads strided over generator calls.  L = table lookups per shot, tied to
// the rank: a 32-bit output word serves S = 4 / 2 / 1 shots (8-, 16-, 32-bit
// fields, low bits first) at rank <= 8 / <= 16 / above, so call g (counter
// (g, variant, fragment, problem)) serves shots 4 S g .. 4 S g + 4 S - 1,
// word j field h being shot (4 g + j) S + h.  fn receives the shot's rank
// coefficient bits.
template <int L, class Fn>
__device__ __forceinline__ void for_shots(uint32_t t0, uint32_t t1, uint4 ctr, const PhiloxKeys& K, uint32_t cmask,
                                          Fn fn) {
  constexpr int S = L == 1 ? 4 : L == 2 ? 2 : 1, WB = 32 / S;
  for (uint32_t g = t0 / (4 * S) + threadIdx.x; (unsigned long long)(4 * S) * g < t1; g += blockDim.x) {
    ctr.x = g;
    const uint4 o = philox4x32_10(ctr, K);
    const uint32_t w4[4] = {o.x, o.y, o.z, o.w};
    if ((unsigned long long)(4 * S) * (g + 1) <= t1) {    // every shot of the call is in range
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int h = 0; h < S; ++h) fn((S == 1 ? w4[j] : w4[j] >> (h * WB)) & cmask);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int h = 0; h < S; ++h) {
          const uint32_t t = (4 * g + j) * S + h;
          if (t < t1) fn((S == 1 ? w4[j] : w4[j] >> (h * WB)) & cmask);
        }
    }
  }
}

// Outcome of coefficient bits c: off ^ the basis vectors c selects.
template <int L>
__device__ __forceinline__ uint32_t space_point(const uint32_t (*tbl)[256], uint32_t off, uint32_t c) {
  uint32_t y = off ^ tbl[0][c & 255];
  if (L >= 2) y ^= tbl[1][(c >> 8) & 255];
  if (L >= 3) y ^= tbl[2][(c >> 16) & 255];
  return y;
}

// A full-rank space in canonical form (pivots = lowest bits, reduced, offset
// with every pivot bit clear) has the identity basis and a zero offset, so a
// shot's outcome is its coefficient bits; checked, not assumed.
__device__ __forceinline__ bool space_is_identity(const SpaceRec& sp, int rank, int nA) {
  if (rank != nA || sp.off != 0u) return false;
  for (int j = 0; j < rank; ++j)
    if (sp.basis[j] != (1u << j)) return false;
  return true;
}

// Calls fn with the lookups a rank needs as a compile-time constant.
template <class Fn>
__device__ __forceinline__ void by_rank(int rank, Fn fn) {
  if (rank <= 8) fn(std::integral_constant<int, 1>{});
  else if (rank <= 16) fn(std::integral_constant<int, 2>{});
  else fn(std::integral_constant<int, 3>{});
}

}  // namespace

constexpr int kHistSmem = 8192;   // dense per-CTA histogram up to |A| = 13

__global__ void __launch_bounds__(256) sample_kernel(DevPlan P, DevRes R, EvalParams E, const int2* items, int spc,
                                                     int chunks) {
  __shared__ uint32_t tbl[3][256];
  __shared__ uint32_t hist[kHistSmem];
  const int item = blockIdx.x / chunks, chunk = blockIdx.x % chunks;
  const int2 it = items[item];
  const FragDev& F = P.frags[it.x];
  const int v = it.y;
  const SpaceRec& sp = R.spaces[F.space_off + v];
  const int rank = sp.rank, nA = F.nA;
  const uint32_t off = sp.off;
  build_tables(tbl, sp, rank);
  const bool smem_hist = (1 << nA) <= kHistSmem;
  if (smem_hist)
    for (int y = threadIdx.x; y < (1 << nA); y += blockDim.x) hist[y] = 0;
  __syncthreads();
  uint32_t* gcounts = R.counts + F.counts_off + ((long long)v << nA);
  const uint32_t cmask = rank >= 32 ? 0xffffffffu : ((1u << rank) - 1u);
  // this CTA's chunk of shots (spc is a multiple of 16: whole generator calls)
  const uint32_t t0 = (uint32_t)chunk * (uint32_t)spc;
  const uint32_t s_end = min((uint32_t)E.shots, t0 + (uint32_t)spc);
  const uint4 ctr = make_uint4(0u, (uint32_t)v, (uint32_t)F.findex, (uint32_t)F.problem);
  by_rank(rank, [&](auto lk) {
    constexpr int L = decltype(lk)::value;
    for_shots<L>(t0, s_end, ctr, E.keys, cmask, [&](uint32_t c) {
      const uint32_t y = space_point<L>(tbl, off, c);
      if (smem_hist) atomicAdd(&hist[y], 1u);
      else atomicAdd(&gcounts[y], 1u);
    });
  });
  if (smem_hist) {
    __syncthreads();
    for (int y = threadIdx.x; y < (1 << nA); y += blockDim.x)
      if (hist[y]) atomicAdd(&gcounts[y], hist[y]);
  }
}

namespace {
// Stores of the hub operand: signed count sums (row index idx = D M + o),
// as 16-bit integers when QH is set (exact: |sum| <= shots <= 32767; the
// readers scale by 1/shots), else scaled to FP32 in QT.
__device__ __forceinline__ void put1(float* QT, int16_t* QH, long long idx, int a, float inv) {
  if (QH) QH[idx] = (int16_t)a;
  else QT[idx] = (float)a * inv;
}
__device__ __forceinline__ void put2(float* QT, int16_t* QH, long long idx, int a, int b, float inv) {
  if (QH) *reinterpret_cast<short2*>(QH + idx) = make_short2((short)a, (short)b);
  else *reinterpret_cast<float2*>(QT + idx) = make_float2((float)a * inv, (float)b * inv);
}
__device__ __forceinline__ void put4(float* QT, int16_t* QH, long long idx, const int (&v)[4], float inv) {
  if (QH) *reinterpret_cast<short4*>(QH + idx) = make_short4((short)v[0], (short)v[1], (short)v[2], (short)v[3]);
  else *reinterpret_cast<float4*>(QT + idx) = make_float4((float)v[0] * inv, (float)v[1] * inv, (float)v[2] * inv,
                                                          (float)v[3] * inv);
}
// signed sums of the counts c[b] (b = output bits) for every sign mask by a
// 16-point Walsh-Hadamard transform, for the outputs o and o+1 (a, c), then
// the variant's operand rows Q^T[D][o..o+1]
__device__ __forceinline__ void hub_pair_out(int (&a)[16], int (&c)[16], int* wht, const int* s_czD,
                                             const int* s_czS, int nz, float* QT, int16_t* QH, int M, int o,
                                             float inv) {
#pragma unroll
  for (int h = 1; h < 16; h <<= 1)
#pragma unroll
    for (int b = 0; b < 16; ++b)
      if (!(b & h)) {
        const int x0 = a[b], y0 = a[b | h], x1 = c[b], y1 = c[b | h];
        a[b] = x0 + y0;
        a[b | h] = x0 - y0;
        c[b] = x1 + y1;
        c[b | h] = x1 - y1;
      }
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    wht[b] = a[b];
    wht[16 + b] = c[b];
  }
  for (int cz = 0; cz < (1 << nz); ++cz) {
    const int sm = s_czS[cz];
    put2(QT, QH, (long long)s_czD[cz] * M + o, wht[sm], wht[16 + sm], inv);
  }
}
// Register select p[i] for a CTA-uniform index (a binary tree of selects).
__device__ __forceinline__ unsigned pick16(const unsigned (&p)[16], int i) {
  unsigned a[8], b[4], c[2];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (i & 1) ? p[2 * k + 1] : p[2 * k];
#pragma unroll
  for (int k = 0; k < 4; ++k) b[k] = (i & 2) ? a[2 * k + 1] : a[2 * k];
#pragma unroll
  for (int k = 0; k < 2; ++k) c[k] = (i & 4) ? b[2 * k + 1] : b[2 * k];
  return (i & 8) ? c[1] : c[0];
}

// Packed variant of hub_pair_out: p[b] holds the counts of outputs o and o+1
// for basis outcome b as two 16-bit lanes; the 16-point transform runs on
// both lanes at once (an output's bins sum to at most the shots, so every
// transform value fits a signed 16-bit lane below 32768 shots), and the
// variant's sign masks pick from registers (no shared-memory scratch).
__device__ __forceinline__ void hub_pair_out_packed(unsigned (&p)[16], const int* s_czD, const int* s_czS, int nz,
                                                    float* QT, int16_t* QH, int M, int o, float inv) {
#pragma unroll
  for (int h = 1; h < 16; h <<= 1)
#pragma unroll
    for (int b = 0; b < 16; ++b)
      if (!(b & h)) {
        const unsigned x = p[b], y = p[b | h];
        p[b] = __vadd2(x, y);
        p[b | h] = __vsub2(x, y);
      }
  for (int cz = 0; cz < (1 << nz); ++cz) {
    const unsigned w = pick16(p, s_czS[cz]);
    const int lo = (int)(short)(w & 0xffffu), hi = (int)(short)(w >> 16);
    put2(QT, QH, (long long)s_czD[cz] * M + o, lo, hi, inv);
  }
}

// The same readout specialised on Q = the quantum outputs (2^Q bins, all
// loaded; the Walsh-Hadamard transform has Q stages): whole-word adds, since
// p = lo + 2^16 hi with |lo|, |hi| <= shots < 2^15 at every stage keeps both
// lanes recoverable (the low lane's borrow is undone when the pair is
// written), and the variant's sign masks (bits < Q) pick by a select tree.
template <int Q>
__device__ __forceinline__ void hub16_readout(const uint32_t* __restrict__ hist2, int m, int M, const int* s_czD,
                                              const int* s_czS, int nz, float* QT, int16_t* QH, float inv) {
  constexpr int NB = 1 << Q;
  for (int o2 = threadIdx.x; o2 < (M >> 1); o2 += blockDim.x) {
    const int o = 2 * o2;
    unsigned p[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) p[b] = hist2[((uint32_t)o | ((uint32_t)b << m)) >> 1];
#pragma unroll
    for (int h = 1; h < NB; h <<= 1)
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (!(b & h)) {
          const unsigned x = p[b], y = p[b | h];
          p[b] = x + y;
          p[b | h] = x - y;
        }
    for (int cz = 0; cz < (1 << nz); ++cz) {
      const int sm = s_czS[cz];
      unsigned t[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) t[b] = p[b];
#pragma unroll
      for (int lvl = 0; lvl < Q; ++lvl)
#pragma unroll
        for (int b = 0; b < (NB >> (lvl + 1)); ++b) t[b] = ((sm >> lvl) & 1) ? t[2 * b + 1] : t[2 * b];
      const unsigned w = t[0] + ((t[0] & 0x8000u) << 1);      // the int16 pair (o, o+1)
      const long long idx = (long long)s_czD[cz] * M + o;
      if (QH) *reinterpret_cast<unsigned*>(QH + idx) = w;
      else put2(QT, nullptr, idx, (int)(short)(w & 0xffffu), (int)(short)(w >> 16), inv);
    }
  }
}

}  // namespace

// The operand rows a hub variant v owns: its preparation digits at the input
// slots, and at the output slots the Pauli its basis reads (X, Y), or I or Z
// for a Z-basis output; one row per choice of I/Z (2^nz rows, bit i of the
// row index = the i-th Z-basis output).  s_czD[row] = the row's Pauli index
// D, s_czS[row] = its sign mask over the quantum-output bits (X/Y-basis
// outputs always flip the sign, a Z-basis output where it reads Z).
// s_nzm[0] = nz, s_nzm[1] = the Z-basis outputs as a bit mask.  Warp 0
// computes them (its lanes < 2^nz write the rows); the caller synchronises
// the block before reading them.
__device__ __forceinline__ void hub_variant_rows(const FragDev& F, int v, int* s_czD, int* s_czS, int* s_nzm) {
  if (threadIdx.x >= 32) return;
  int beta[kMaxCuts], zpos[kMaxCuts], zout[kMaxCuts];
  int nz, zm;
  int t = v;
  for (int i = 0; i < F.qin; ++i) t /= 4;
  for (int j = 0; j < F.qout; ++j) { beta[j] = t % 3; t /= 3; }
  int Dbase = 0, fixed_mask = 0;
  nz = 0;
  zm = 0;
  for (int j = 0; j < F.n_slots; ++j) {
    const int code = F.slot_code[j], idx = code & 255;
    if ((code >> 8) == 0) {
      int u = v;
      for (int i = 0; i < idx; ++i) u /= 4;
      Dbase |= (u % 4) << (2 * j);
    } else if (beta[idx] == 2) {
      zpos[nz] = j;
      zout[nz++] = idx;
      zm |= 1 << idx;
    } else {
      Dbase |= (beta[idx] == 0 ? 1 : 2) << (2 * j);
      fixed_mask |= 1 << idx;
    }
  }
  if ((int)threadIdx.x < (1 << nz)) {
    int D = Dbase, smask = fixed_mask;
    for (int i = 0; i < nz; ++i)
      if ((threadIdx.x >> i) & 1) { D |= 3 << (2 * zpos[i]); smask |= 1 << zout[i]; }
    s_czD[threadIdx.x] = D;
    s_czS[threadIdx.x] = smask;
  }
  if (threadIdx.x == 0) {
    s_nzm[0] = nz;
    s_nzm[1] = zm;
  }
}

// --- K3 + K5 fused for the hub of a star --------------------------------
// One CTA per hub variant: all its shots into a shared-memory histogram
// (16-bit counters packed in pairs, so |A| <= 16 fits 128 KB), then the
// variant's slice of the hub operand
//   Q[o, (s, P_out)] = sum_b prod_j lambda(P_out_j, b_j) count(o, b) / shots
// for every P_out with beta(P_out) = the variant's bases, written to the
// transposed store Q^T.  Dense counts are written only when kept for
// inspection.
__global__ void __launch_bounds__(512) sample_hub_kernel(DevPlan P, DevRes R, EvalParams E, const int2* items,
                                                         int keep_counts, int wide, int hist_words) {
  extern __shared__ __align__(16) uint32_t hist2[];
  __shared__ uint32_t tbl[3][256];
  __shared__ FragDev sF;
  __shared__ int s_czD[16], s_czS[16], s_nzm[2], s_ident;
  const int2 it = items[blockIdx.x];
  {
    const int* src = reinterpret_cast<const int*>(P.frags + it.x);
    int* dst = reinterpret_cast<int*>(&sF);
    for (int i = threadIdx.x; i < (int)(sizeof(FragDev) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const FragDev& F = sF;
  const int v = it.y, nA = F.nA;
  const SpaceRec& sp = R.spaces[F.space_off + v];
  const int rank = sp.rank;
  const uint32_t off = sp.off;
  if (threadIdx.x == 32) s_ident = space_is_identity(sp, rank, nA) ? 1 : 0;
  if (F.qout <= 4) hub_variant_rows(F, v, s_czD, s_czS, s_nzm);   // warp 0: at most 16 rows
  __syncthreads();
  if (!s_ident) build_tables(tbl, sp, rank);   // a full-rank space needs no lookup tables
  const int nwords = wide ? (1 << nA) : ((1 << nA) > 1 ? (1 << (nA - 1)) : 1);
  {   // zero the histogram, 16 bytes per store
    uint4* h4 = reinterpret_cast<uint4*>(hist2);
    for (int i = threadIdx.x; i < nwords / 4; i += blockDim.x) h4[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = 4 * (nwords / 4) + threadIdx.x; i < nwords; i += blockDim.x) hist2[i] = 0u;
  }
  __syncthreads();
  const bool ident = s_ident != 0;
  const uint32_t cmask = rank >= 32 ? 0xffffffffu : ((1u << rank) - 1u);
  {
    const uint4 ctr = make_uint4(0u, (uint32_t)v, (uint32_t)F.findex, (uint32_t)F.problem);
    by_rank(rank, [&](auto lk) {
      constexpr int L = decltype(lk)::value;
      for_shots<L>(0u, E.shots, ctr, E.keys, cmask, [&](uint32_t c) {
        const uint32_t y = ident ? c : space_point<L>(tbl, off, c);   // full rank: the coefficient bits
        if (wide) atomicAdd(&hist2[y], 1u);
        else atomicAdd(&hist2[y >> 1], 1u << ((y & 1u) << 4));
      });
    });
  }
  __syncthreads();
  auto count = [&](uint32_t y) -> uint32_t {
    return wide ? hist2[y] : (hist2[y >> 1] >> ((y & 1u) << 4)) & 0xffffu;
  };
  if (keep_counts) {
    uint32_t* g = R.counts + F.counts_off + ((long long)v << nA);
    for (uint32_t y = threadIdx.x; y < (1u << nA); y += blockDim.x) g[y] = count(y);
  }
  // Q is stored transposed, Q^T[D][o] (o fastest), so each D of the variant
  // is one coalesced row of 2^m floats.
  const int m = F.m, M = 1 << m, nb = 1 << F.qout;
  const float inv = (float)E.inv_shots;
  float* QT = R.TQ + F.T_off;
  int16_t* QH = R.hub_i16 ? reinterpret_cast<int16_t*>(R.TQ + F.T_off) : nullptr;
  if (!wide && m >= 1 && F.qout <= 4 && E.shots <= (1u << 26)) {
    // Pairs of outputs (o, o+1) share the packed counter words.  Per pair,
    // a 16-point Walsh-Hadamard transform over the output bits gives the
    // signed sum for every sign mask at once; each thread parks it in its
    // own 33-word slot after the histogram (odd stride: no bank conflicts)
    // and picks the variant's masks; below 32768 shots the transform runs
    // on packed lanes and picks from registers, with no slot.
    const int nz = s_nzm[0];
    int* wht = reinterpret_cast<int*>(hist2 + hist_words) + threadIdx.x * (E.shots <= 32767u ? 0 : 33);
    if (E.shots <= 32767u) {
      // an output's bins sum to at most the shots, so every transform value
      // fits a signed 16-bit lane: the counter word (outputs o, o+1) is
      // transformed as is, two outputs per SIMD add
      switch (F.qout) {
        case 0: hub16_readout<0>(hist2, m, M, s_czD, s_czS, nz, QT, QH, inv); break;
        case 1: hub16_readout<1>(hist2, m, M, s_czD, s_czS, nz, QT, QH, inv); break;
        case 2: hub16_readout<2>(hist2, m, M, s_czD, s_czS, nz, QT, QH, inv); break;
        case 3: hub16_readout<3>(hist2, m, M, s_czD, s_czS, nz, QT, QH, inv); break;
        default: hub16_readout<4>(hist2, m, M, s_czD, s_czS, nz, QT, QH, inv); break;
      }
    } else
    for (int o2 = threadIdx.x; o2 < (M >> 1); o2 += blockDim.x) {
      const int o = 2 * o2;
      int a[16], c[16];
#pragma unroll
      for (int b = 0; b < 16; ++b) {
        const uint32_t w = b < nb ? hist2[((uint32_t)o | ((uint32_t)b << m)) >> 1] : 0u;
        a[b] = (int)(w & 0xffffu);
        c[b] = (int)(w >> 16);
      }
#pragma unroll
      for (int h = 1; h < 16; h <<= 1)
#pragma unroll
        for (int b = 0; b < 16; ++b)
          if (!(b & h)) {
            const int x0 = a[b], y0 = a[b | h], x1 = c[b], y1 = c[b | h];
            a[b] = x0 + y0;
            a[b | h] = x0 - y0;
            c[b] = x1 + y1;
            c[b | h] = x1 - y1;
          }
#pragma unroll
      for (int b = 0; b < 16; ++b) {
        wht[b] = a[b];
        wht[16 + b] = c[b];
      }
      for (int cz = 0; cz < (1 << nz); ++cz) {
        const int sm = s_czS[cz];
        put2(QT, QH, (long long)s_czD[cz] * M + o, wht[sm], wht[16 + sm], inv);
      }
    }
  } else if (F.qout <= 4 && E.shots <= (1u << 26)) {     // |acc| <= 16 shots fits an int
    const int nz = s_nzm[0];
    for (int o = threadIdx.x; o < M; o += blockDim.x) {
      int c[16];
#pragma unroll
      for (int b = 0; b < 16; ++b) c[b] = b < nb ? (int)count((uint32_t)o | ((uint32_t)b << m)) : 0;
      for (int cz = 0; cz < (1 << nz); ++cz) {
        const int D = s_czD[cz], smask = s_czS[cz];
        int acc = 0;
#pragma unroll
        for (int b = 0; b < 16; ++b) acc += (__popc(b & smask) & 1) ? -c[b] : c[b];
        put1(QT, QH, (long long)D * M + o, acc, inv);
      }
    }
  } else {   // more than four quantum outputs: the variant's digits decoded per thread
    int beta[kMaxCuts];
    {
      int t = v;
      for (int i = 0; i < F.qin; ++i) t /= 4;
      for (int j = 0; j < F.qout; ++j) { beta[j] = t % 3; t /= 3; }
    }
    int zpos[kMaxCuts], zout[kMaxCuts], nz = 0;
    int Dbase = 0, fixed_mask = 0;   // fixed_mask: X/Y-basis outputs, whose outcome always flips the sign
    for (int j = 0; j < F.n_slots; ++j) {
      const int code = F.slot_code[j], idx = code & 255;
      if ((code >> 8) == 0) {
        int t = v;
        for (int i = 0; i < idx; ++i) t /= 4;
        Dbase |= (t % 4) << (2 * j);
      } else if (beta[idx] == 2) {
        zpos[nz] = j;                           // Z basis: P_out in {I, Z}
        zout[nz++] = idx;
      } else {
        Dbase |= (beta[idx] == 0 ? 1 : 2) << (2 * j);   // X basis -> X, Y basis -> Y
        fixed_mask |= 1 << idx;
      }
    }
    for (int cz = 0; cz < (1 << nz); ++cz) {
      int D = Dbase, smask = fixed_mask;
      for (int i = 0; i < nz; ++i)
        if ((cz >> i) & 1) { D |= 3 << (2 * zpos[i]); smask |= 1 << zout[i]; }
      for (int o = threadIdx.x; o < M; o += blockDim.x) {
        long long acc = 0;
        for (int b = 0; b < nb; ++b) {
          const long long cnt = count((uint32_t)o | ((uint32_t)b << m));
          acc += (__popc(b & smask) & 1) ? -cnt : cnt;
        }
        if (QH) QH[(long long)D * M + o] = (int16_t)acc;
        else QT[(long long)D * M + o] = (float)((double)acc * E.inv_shots);
      }
    }
  }
}

// Readout of a byte-counter histogram into the variant's operand rows,
// specialised on ZM, the quantum outputs measured in the Z basis.  Row cz
// of the variant needs S(o, cz) = sum_b (-1)^(b . smask_cz) count(o, b) with
// smask_cz = the X/Y-basis outputs (whose outcome always flips the sign)
// plus the Z outputs selected by cz.  So the bins are first summed over the
// X/Y bits with their fixed signs (F over the Z bits), then a Walsh-Hadamard
// transform over the Z bits gives every row at once: 16 - 2^nz + nz 2^nz
// adds instead of a full 16-point transform.  Four outputs o..o+3 share a
// counter word; each half is processed as two 16-bit lanes of one 32-bit
// integer (signed lane sums stay below 2^15 in magnitude, so plain integer
// adds keep the lanes separable).  Returns the thread's sum of all counter
// bytes read (the caller compares the block's total with the shots: a byte
// that wrapped makes it smaller).
__host__ __device__ constexpr int popc4(int x) { return (x & 1) + ((x >> 1) & 1) + ((x >> 2) & 1) + ((x >> 3) & 1); }
__host__ __device__ constexpr int pext4(int b, int zm) {
  int r = 0, k = 0;
  for (int j = 0; j < 4; ++j)
    if ((zm >> j) & 1) r |= ((b >> j) & 1) << k++;
  return r;
}

template <int ZM>
__device__ __forceinline__ unsigned hub8_readout(const uint32_t* __restrict__ h32, int m, int M, int nb,
                                                 const int* s_czD, float* __restrict__ QT, int16_t* __restrict__ QH,
                                                 float inv) {
  constexpr int NR = 1 << popc4(ZM);
  unsigned tot = 0;
  for (int q = threadIdx.x; q < (M >> 2); q += blockDim.x) {
    const int o = 4 * q;
    uint32_t w[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) w[b] = b < nb ? h32[((uint32_t)o | ((uint32_t)b << m)) >> 2] : 0u;
#pragma unroll
    for (int b = 0; b < 16; ++b) tot = __dp4a(w[b], 0x01010101u, tot);
    uint32_t W[NR][2];     // per row: outputs (o, o+1) and (o+2, o+3) as int16 pairs
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      int F[NR];
#pragma unroll
      for (int i = 0; i < NR; ++i) F[i] = 0;
#pragma unroll
      for (int b = 0; b < 16; ++b) {     // outputs o + 2 half, o + 2 half + 1 as 16-bit lanes
        const int x = (int)__byte_perm(w[b], 0u, half ? 0x4342 : 0x4140);
        if (popc4(b & ~ZM & 15) & 1) F[pext4(b, ZM)] -= x;
        else F[pext4(b, ZM)] += x;
      }
#pragma unroll
      for (int h = 1; h < NR; h <<= 1)
#pragma unroll
        for (int i = 0; i < NR; ++i)
          if (!(i & h)) {
            const int a = F[i], c = F[i | h];
            F[i] = a + c;
            F[i | h] = a - c;
          }
      // F = lo + 2^16 hi with |lo|, |hi| <= 16 x 255: the int16 pair word is
      // F plus the borrow its low lane took from the high one
#pragma unroll
      for (int i = 0; i < NR; ++i) W[i][half] = (uint32_t)F[i] + (((uint32_t)F[i] & 0x8000u) << 1);
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const long long idx = (long long)s_czD[i] * M + o;
      if (QH) {
        *reinterpret_cast<uint2*>(QH + idx) = make_uint2(W[i][0], W[i][1]);
      } else {
        const int v[4] = {(int)(short)(W[i][0] & 0xffffu), (int)(short)(W[i][0] >> 16),
                          (int)(short)(W[i][1] & 0xffffu), (int)(short)(W[i][1] >> 16)};
        put4(QT, nullptr, idx, v, inv);
      }
    }
  }
  return tot;
}

// --- the hub sampler with byte counters (three CTAs per SM) ---------------
// Same result as sample_hub_kernel, for hubs with |A| <= 16, at least two
// marginal bits and at most four quantum outputs, below 65536 shots.  The
// histogram holds 8-bit counters (2^16 of them in 64 KB) so three CTAs fit
// on an SM (a readout sum of 16 bytes stays below 2^15 whatever the shots).  Counts stay exact: a variant whose expected count per outcome
// is above 64 (shots > 64 * 2^rank), or whose counting wrapped a byte (the
// bytes then sum to less than the shots: a wrap loses 256 from the byte and
// carries at most 1 into the next), is counted again with 16-bit counters
// in two passes, each over the outputs o of one half (top marginal bit),
// and its operand rows are rewritten.
template <int NT>    // 256 threads (three CTAs per SM) or 512 (two): registers for each
__global__ void __launch_bounds__(NT, NT >= 512 ? 2 : 3) sample_hub8_kernel(DevPlan P, DevRes R, EvalParams E,
                                                                          const int2* items, int keep_counts,
                                                                          int hist_words) {
  extern __shared__ __align__(16) uint32_t h32[];
  __shared__ uint32_t tbl[3][256];
  __shared__ FragDev sF;
  __shared__ int s_czD[16], s_czS[16], s_nzm[2];
  __shared__ unsigned s_tot;
  __shared__ int s_ident;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int2 it = items[blockIdx.x];
  {
    const int* src = reinterpret_cast<const int*>(P.frags + it.x);
    int* dst = reinterpret_cast<int*>(&sF);
    for (int i = tid; i < (int)(sizeof(FragDev) / 4); i += nt) dst[i] = src[i];
  }
  if (tid == 0) s_tot = 0u;
  __syncthreads();
  const FragDev& F = sF;
  const int v = it.y, nA = F.nA, m = F.m, M = 1 << m, nb = 1 << F.qout;
  const SpaceRec& sp = R.spaces[F.space_off + v];
  const int rank = sp.rank;
  const uint32_t off = sp.off;
  if (tid == 32) s_ident = space_is_identity(sp, rank, nA) ? 1 : 0;
  // the variant's operand rows: one D and sign mask per Z-basis choice
  hub_variant_rows(F, v, s_czD, s_czS, s_nzm);
  __syncthreads();
  const bool ident = s_ident != 0;
  if (!ident) build_tables(tbl, sp, rank);   // a full-rank space needs no lookup tables
  const uint32_t cmask = rank >= 32 ? 0xffffffffu : ((1u << rank) - 1u);
  const float inv = (float)E.inv_shots;
  float* QT = R.TQ + F.T_off;
  int16_t* QH = R.hub_i16 ? reinterpret_cast<int16_t*>(R.TQ + F.T_off) : nullptr;
  const int wstride = E.shots <= 32767u ? 0 : 33;    // only the unpacked transform parks values
  int* wht = reinterpret_cast<int*>(h32 + hist_words) + tid * wstride;
  uint32_t* gcount = R.counts + F.counts_off + ((long long)v << nA);
  bool narrow = (unsigned long long)E.shots <= (64ull << rank);
  if (narrow) {
    {   // zero the histogram, 16 bytes per store
      uint4* h4 = reinterpret_cast<uint4*>(h32);
      for (int i = tid; i < (1 << nA) / 16; i += nt) h4[i] = make_uint4(0u, 0u, 0u, 0u);
      for (int i = 4 * ((1 << nA) / 16) + tid; i < (1 << nA) / 4; i += nt) h32[i] = 0u;
    }
    __syncthreads();
    const uint4 ctr = make_uint4(0u, (uint32_t)v, (uint32_t)F.findex, (uint32_t)F.problem);
    by_rank(rank, [&](auto lk) {
      constexpr int L = decltype(lk)::value;
      if (ident)        // full rank: the outcome is the coefficient bits (no table lookup)
        for_shots<L>(0u, E.shots, ctr, E.keys, cmask,
                     [&](uint32_t c) { atomicAdd(&h32[c >> 2], 1u << ((c & 3u) << 3)); });
      else
        for_shots<L>(0u, E.shots, ctr, E.keys, cmask, [&](uint32_t c) {
          const uint32_t y = space_point<L>(tbl, off, c);
          atomicAdd(&h32[y >> 2], 1u << ((y & 3u) << 3));
        });
    });
    __syncthreads();
    if (keep_counts)
      for (uint32_t y = tid; y < (1u << nA); y += nt) gcount[y] = (h32[y >> 2] >> ((y & 3u) << 3)) & 0xffu;
    unsigned tot = 0;
    switch (s_nzm[1]) {
#define CCS_HUB8_CASE(z) \
  case z: tot = hub8_readout<z>(h32, m, M, nb, s_czD, QT, QH, inv); break;
      CCS_HUB8_CASE(0) CCS_HUB8_CASE(1) CCS_HUB8_CASE(2) CCS_HUB8_CASE(3)
      CCS_HUB8_CASE(4) CCS_HUB8_CASE(5) CCS_HUB8_CASE(6) CCS_HUB8_CASE(7)
      CCS_HUB8_CASE(8) CCS_HUB8_CASE(9) CCS_HUB8_CASE(10) CCS_HUB8_CASE(11)
      CCS_HUB8_CASE(12) CCS_HUB8_CASE(13) CCS_HUB8_CASE(14) CCS_HUB8_CASE(15)
#undef CCS_HUB8_CASE
      default: break;
    }
    tot = __reduce_add_sync(0xffffffffu, tot);
    if ((tid & 31) == 0) atomicAdd(&s_tot, tot);
    __syncthreads();
    narrow = s_tot == E.shots;      // no byte wrapped
  }
  if (!narrow) {   // 16-bit counters, outputs of one half (top marginal bit) per pass
    __syncthreads();
    const int nz = s_nzm[0];
    const int mh = m - 1, Mh = M >> 1;
    for (int h = 0; h < 2; ++h) {
      __syncthreads();
      for (int i = tid; i < (1 << (nA - 1)) / 2; i += nt) h32[i] = 0u;
      __syncthreads();
      const uint4 ctr = make_uint4(0u, (uint32_t)v, (uint32_t)F.findex, (uint32_t)F.problem);
      by_rank(rank, [&](auto lk) {
        constexpr int L = decltype(lk)::value;
        for_shots<L>(0u, E.shots, ctr, E.keys, cmask, [&](uint32_t c) {
          const uint32_t y = ident ? c : space_point<L>(tbl, off, c);
          if ((int)((y >> mh) & 1u) != h) return;
          const uint32_t yh = (y & (uint32_t)(Mh - 1)) | ((y >> m) << mh);
          atomicAdd(&h32[yh >> 1], 1u << ((yh & 1u) << 4));
        });
      });
      __syncthreads();
      if (keep_counts)
        for (uint32_t yh = tid; yh < (1u << (nA - 1)); yh += nt) {
          const uint32_t y = (yh & (uint32_t)(Mh - 1)) | ((uint32_t)h << mh) | ((yh >> mh) << m);
          gcount[y] = (h32[yh >> 1] >> ((yh & 1u) << 4)) & 0xffffu;
        }
      for (int o2 = tid; o2 < (Mh >> 1); o2 += nt) {    // pairs of outputs within the half
        const int ol = 2 * o2;
        if (wstride == 0) {                    // an output's bins sum to at most the shots
          unsigned pk[16];
#pragma unroll
          for (int b = 0; b < 16; ++b) pk[b] = b < nb ? h32[((uint32_t)ol | ((uint32_t)b << mh)) >> 1] : 0u;
          hub_pair_out_packed(pk, s_czD, s_czS, nz, QT, QH, M, h * Mh + ol, inv);
          continue;
        }
        int a[16], c[16];
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          const uint32_t w = b < nb ? h32[((uint32_t)ol | ((uint32_t)b << mh)) >> 1] : 0u;
          a[b] = (int)(w & 0xffffu);
          c[b] = (int)(w >> 16);
        }
        hub_pair_out(a, c, wht, s_czD, s_czS, nz, QT, QH, M, h * Mh + ol, inv);
      }
    }
  }
}

// --- stitched mode: a Clifford hub's operand in closed form (Sec. IX) -------
// A variant's outcomes y = (o, b) (o the marginal bits, b the quantum-output
// bits) are uniform, probability 2^-r, on off + span(B), B in reduced
// echelon form with pivot = lowest bit.  The vectors with pivot in b have no
// o part: they span K = {b : (0, b) in span B}, 2^kb elements.  The others
// project to an echelon basis of the o-projection.  For an output o in
// off_o + that projection the b with (o, b) in the space form a coset
// b0(o) + K, with b0(o) = off_b + the b parts of the vectors o's pivot bits
// select; for other o there is none.  So row cz of the operand,
//   Q(o, cz) = sum_b (-1)^(b . s_cz) p(o, b),
// vanishes for every o unless s_cz is orthogonal to K, and is then
// 2^(kb - r) (-1)^(b0(o) . s_cz) on the projection and 0 elsewhere: exact
// in FP32, no shots, no per-variant distribution.  One CTA per hub variant
// writes its rows' flags (1 unless identically zero) and its nonzero rows;
// its zero rows only when the problem's contraction reads every row (the
// streaming GEMM skips flagged rows).
__global__ void __launch_bounds__(256) hub_exact_kernel(DevPlan P, DevRes R, const int2* items) {
  __shared__ FragDev sF;
  __shared__ int s_czD[16], s_czS[16], s_live[16], s_nzm[2];
  __shared__ uint32_t s_vo[kMaxMeas], s_vb[kMaxMeas], s_kg[kMaxMeas];
  __shared__ int s_piv[kMaxMeas], s_cnt[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int2 it = items[blockIdx.x];
  {
    const int* src = reinterpret_cast<const int*>(P.frags + it.x);
    int* dst = reinterpret_cast<int*>(&sF);
    for (int i = tid; i < (int)(sizeof(FragDev) / 4); i += nt) dst[i] = src[i];
  }
  __syncthreads();
  const FragDev& F = sF;
  const int v = it.y, m = F.m, M = 1 << m;
  hub_variant_rows(F, v, s_czD, s_czS, s_nzm);
  const SpaceRec& sp = R.spaces[F.space_off + v];
  const int rank = sp.rank;
  if (tid == 32) {
    int ro = 0, kb = 0;
    for (int j = 0; j < rank; ++j) {
      const uint32_t vec = sp.basis[j];
      const int p = __ffs((int)vec) - 1;
      if (p < m) { s_vo[ro] = vec & (uint32_t)(M - 1); s_vb[ro] = vec >> m; s_piv[ro] = p; ++ro; }
      else s_kg[kb++] = vec >> m;
    }
    s_cnt[0] = ro;
    s_cnt[1] = kb;
  }
  __syncthreads();
  const int ro = s_cnt[0], kb = s_cnt[1], nrows = 1 << s_nzm[0];
  if (tid < nrows) {
    bool live = true;
    for (int j = 0; j < kb; ++j) live = live && !(__popc(s_kg[j] & (uint32_t)s_czS[tid]) & 1);
    s_live[tid] = live ? 1 : 0;
    R.qnz[F.qrow_off + s_czD[tid]] = live ? 1 : 0;
  }
  __syncthreads();
  const bool write_zero = P.problems[F.problem].stream == 0;
  int any = write_zero ? 1 : 0;
  for (int i = 0; i < nrows; ++i) any |= s_live[i];
  if (!any) return;
  const float c = ldexpf(1.0f, kb - rank);
  const uint32_t off_o = sp.off & (uint32_t)(M - 1), off_b = sp.off >> m;
  float* QT = R.TQ + F.T_off;
  for (int o = tid; o < M; o += nt) {
    const uint32_t y = (uint32_t)o ^ off_o;
    uint32_t x = 0u, bb = off_b;
    for (int t = 0; t < ro; ++t)
      if ((y >> s_piv[t]) & 1u) { x ^= s_vo[t]; bb ^= s_vb[t]; }
    const bool member = x == y;
    for (int cz = 0; cz < nrows; ++cz) {
      if (!s_live[cz] && !write_zero) continue;
      const float val = (s_live[cz] && member) ? ((__popc(bb & (uint32_t)s_czS[cz]) & 1) ? -c : c) : 0.f;
      QT[(long long)s_czD[cz] * M + o] = val;
    }
  }
}

cudaError_t launch_hub_exact(const DevPlan& p, const DevRes& r, const int2* items, int n_items, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  hub_exact_kernel<<<n_items, 256, 0, s>>>(p, r, items); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sample_hub(const DevPlan& p, const DevRes& r, const EvalParams& e, const int2* items, int n_items,
                              int max_nA, int threads, int keep_counts, bool bytes_ok, cudaStream_t s) {
  if (n_items == 0 || e.shots == 0) return cudaSuccess;
  if (bytes_ok && e.shots <= 0xffffu && max_nA >= 2 && max_nA <= 16) {   // byte counters, 256 or 512 threads
    const int t8 = threads >= 512 ? 512 : 256;
    const int hist_words = (1 << max_nA) / 4;
    const size_t smem = (size_t)4 * hist_words + (size_t)t8 * (e.shots <= 32767u ? 0 : 33) * 4;
    auto kern = t8 == 512 ? sample_hub8_kernel<512> : sample_hub8_kernel<256>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<n_items, t8, smem, s>>>(p, r, e, items, keep_counts, hist_words); note_launch();
    return cudaGetLastError();
  }
  const int wide = e.shots > 0xffffu ? 1 : 0;     // 32-bit counters when 16 bits could overflow
  const int hist_words = wide ? (1 << max_nA) : ((1 << max_nA) > 1 ? (1 << (max_nA - 1)) : 1);
  // packed counters, then 33 ints per thread for the transform of the 16-bit path
  threads = threads >= 512 ? 512 : threads >= 256 ? 256 : 128;
  const size_t smem = (size_t)4 * hist_words + (wide ? 0 : (size_t)threads * (e.shots <= 32767u ? 0 : 33) * 4);
  cudaError_t err = cudaFuncSetAttribute(sample_hub_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  sample_hub_kernel<<<n_items, threads, smem, s>>>(p, r, e, items, keep_counts, wide, hist_words); note_launch();
  return cudaGetLastError();
}

template <int G>
static cudaError_t launch_clifford_g(const DevPlan& p, const DevRes& r, const EvalParams& e, int threads,
                                     int smem_words, int grid, cudaStream_t s) {
  const size_t smem = (size_t)smem_words * 8;
  cudaError_t err = cudaFuncSetAttribute(clifford_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  clifford_kernel<G><<<grid, threads, smem, s>>>(p, r, e, smem_words); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_clifford(const DevPlan& p, const DevRes& r, const EvalParams& e, int threads, int words_per_op,
                            int smem_words, int grid, cudaStream_t s) {
  if (p.n_items_cliff == 0) return cudaSuccess;
  switch (words_per_op) {
    case 8: return launch_clifford_g<8>(p, r, e, threads, smem_words, grid, s);
    case 4: return launch_clifford_g<4>(p, r, e, threads, smem_words, grid, s);
    case 2: return launch_clifford_g<2>(p, r, e, threads, smem_words, grid, s);
    default: return launch_clifford_g<1>(p, r, e, threads, smem_words, grid, s);
  }
}

cudaError_t launch_body(const DevPlan& p, const DevRes& r, int smem_optin, bool basis, cudaStream_t s) {
  if (p.n_items_body == 0) return cudaSuccess;
  const int words = std::max(p.max_body_cols, std::min(p.max_body_stage_words, smem_optin / 8));
  // moments of at most 32 ops (deep, narrow circuits): eight lanes per op,
  // a warp per 4 ops of the widest moment; otherwise one thread per op of the
  // widest moment (whole warps, 32..256): fewer idle warps at each barrier
  const bool coop = p.max_moment_ops <= 32;
  const int threads = coop ? std::max(32, (8 * p.max_moment_ops + 31) / 32 * 32)
                           : std::min(256, std::max(32, (p.max_moment_ops + 31) / 32 * 32));
  auto kern = coop ? body_kernel<true> : body_kernel<false>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, words * 8);
  if (err != cudaSuccess) return err;
  kern<<<p.n_items_body, threads, (size_t)words * 8, s>>>(p, r, words); note_launch();
  err = cudaGetLastError();
  if (!basis) return err;
  if (err != cudaSuccess || p.n_cliff_frags == 0) return err;
  // fragments with no measurement record get no table: nothing reads it
  body_basis_kernel<<<p.n_cliff_frags + p.n_items_zimg, 256, 0, s>>>(p, r); note_launch();
  if ((err = cudaGetLastError()) != cudaSuccess || p.n_items_proj == 0) return err;
  proj_kernel<<<(p.n_items_proj + 7) / 8, 256, 0, s>>>(p, r); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_screen(const DevPlan& p, const DevRes& r, const EvalParams& e, int sm_count, int smem_optin,
                          cudaStream_t s) {
  if (p.n_items_cliff == 0) return cudaSuccess;
  const int warps = 8;
  const long long need = (p.n_items_cliff + warps - 1) / warps;
  const int rank_blocks = (int)(need < (long long)sm_count * 8 ? need : (long long)sm_count * 8);
  const int img = p.n_zblocks ? std::min(p.img_words_max, std::min(4096, smem_optin / 8)) : 0;
  if (img) {
    cudaError_t err = cudaFuncSetAttribute(screen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, img * 8);
    if (err != cudaSuccess) return err;
  }
  screen_kernel<<<rank_blocks + p.n_zblocks, 32 * warps, (size_t)img * 8, s>>>(p, r, e, rank_blocks, img);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sample(const DevPlan& p, const DevRes& r, const EvalParams& e, const int2* items, int n_items,
                          int spc, int threads, cudaStream_t s) {
  if (n_items == 0 || e.shots == 0) return cudaSuccess;
  const int chunks = (int)((e.shots + spc - 1) / spc);
  const long long grid = (long long)n_items * chunks;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  sample_kernel<<<(unsigned)grid, threads, 0, s>>>(p, r, e, items, spc, chunks); note_launch();
  return cudaGetLastError();
}

}  // namespace ccs
