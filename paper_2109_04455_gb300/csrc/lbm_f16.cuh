// FP16-deviation storage (populations stored as half of 2^14 (g - w_i R),
// R the storing node's concentration, itself stored in half): the update of
// an interior node, in a one-node form (used by the batch kernel) and a
// two-node bulk kernel.  Included by lbm_kernels.cuh after AdrArgs and the
// lattice helpers.
#pragma once

namespace lbm {

// ---------------------------------------------------------------------------
// Interior update of the FP16-deviation storage.  The arithmetic runs on the
// populations scaled by 2^14, G = 2^14 g, the scale the deviations are
// stored in, so a stored half converts straight into it; the concentration
// is brought back to scale 1 once per species and node.  Scaling by a power
// of two is exact, so every result equals the unscaled arithmetic's.  Each
// operation is written with an explicit rounding (no contraction left to
// the compiler), so the one-node form (batch kernel) and the two-node form
// (bulk step) give the same bits for the same node.
// ---------------------------------------------------------------------------
namespace f16 {
constexpr float kDown = 1.0f / 16384.0f, kUp = 16384.0f;
__device__ __forceinline__ float w(int i) { return Lattice<float>::w(i); }
// scaled population pulled from a source node: its stored deviation h plus
// w_i 2^14 times the source's reference concentration r (as stored, at
// scale 1).  w_i 2^14 is exact, so this equals fma(w_i, 2^14 r, h) bit for
// bit, without the multiply by 2^14.
__device__ __forceinline__ float pull(int i, float h, float r) {
  return __fmaf_rn(w(i) * kUp, r, h);
}
// equilibrium factors E_i(u) = w_i (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u),
// built for each direction together with its opposite (c.u changes sign,
// the even part w_i (1 + 4.5 (c.u)^2 - 1.5 u.u) is shared)
__device__ __forceinline__ void eq(float ux, float uy, float (&E)[9]) {
  const float base = __fmaf_rn(-1.5f, __fmaf_rn(ux, ux, __fmul_rn(uy, uy)), 1.0f);
  E[0] = __fmul_rn(w(0), base);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = k < 2 ? k + 1 : k + 3;   // 1, 2, 5, 6
    const float cu = __fadd_rn(float(cx(i)) * ux, float(cy(i)) * uy);
    const float even = __fmul_rn(w(i), __fmaf_rn(__fmul_rn(4.5f, cu), cu, base));
    E[i] = __fmaf_rn(3.0f * w(i), cu, even);
    E[opp(i)] = __fmaf_rn(-3.0f * w(i), cu, even);
  }
}
// C_s at scale 2^14: a pairwise sum (short dependency chains)
__device__ __forceinline__ float sum9(const float (&g)[9]) {
  const float a = __fadd_rn(__fadd_rn(g[0], g[1]), __fadd_rn(g[2], g[3]));
  const float b = __fadd_rn(__fadd_rn(g[4], g[5]), __fadd_rn(g[6], g[7]));
  return __fadd_rn(__fadd_rn(a, b), g[8]);
}
// Per node and species: keep = 1 - om, a = om C_s (scale 2^14), and w_i
// times the node's stored reference (scale 2^14) for the three weights.
struct PushK {
  float keep, a, wq[3];
};
__device__ __forceinline__ PushK push_k(float om, float cs, float cqs) {
  PushK k;
  k.keep = __fsub_rn(1.0f, om);
  k.a = __fmul_rn(om, cs);
  k.wq[0] = __fmul_rn(w(0), cqs);
  k.wq[1] = __fmul_rn(w(1), cqs);
  k.wq[2] = __fmul_rn(w(5), cqs);
  return k;
}
// value stored for population i: the BGK relaxation (1 - om) G + om C_s E_i
// less w_i times the node's stored reference, all at scale 2^14: two FMAs
__device__ __forceinline__ float push(int i, float g, float e, const PushK &k) {
  const float wq = i == 0 ? k.wq[0] : (i < 5 ? k.wq[1] : k.wq[2]);
  return __fmaf_rn(k.keep, g, __fmaf_rn(k.a, e, -wq));
}

// Packed two-node forms of the arithmetic above (this part's f32x2 FMA, add
// and multiply): lane 0 is node x0, lane 1 node x0 + 1, and each lane is
// rounded exactly like the scalar operation, so a lane's bits equal the
// one-node form's.  One packed instruction does the work of two (measured
// 0.7% faster per step than the scalar form on two nodes).
__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }
__device__ __forceinline__ void eq2(float2 ux, float2 uy, float2 (&E)[9]) {
  const float2 base = __ffma2_rn(dup(-1.5f), __ffma2_rn(ux, ux, __fmul2_rn(uy, uy)),
                                 dup(1.0f));
  E[0] = __fmul2_rn(dup(w(0)), base);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = k < 2 ? k + 1 : k + 3;   // 1, 2, 5, 6
    const float2 cu = __fadd2_rn(__fmul2_rn(dup(float(cx(i))), ux),
                                 __fmul2_rn(dup(float(cy(i))), uy));
    const float2 even = __fmul2_rn(dup(w(i)), __ffma2_rn(__fmul2_rn(dup(4.5f), cu), cu, base));
    E[i] = __ffma2_rn(dup(3.0f * w(i)), cu, even);
    E[opp(i)] = __ffma2_rn(dup(-3.0f * w(i)), cu, even);
  }
}
__device__ __forceinline__ float2 sum9(const float2 (&g)[9]) {
  const float2 a = __fadd2_rn(__fadd2_rn(g[0], g[1]), __fadd2_rn(g[2], g[3]));
  const float2 b = __fadd2_rn(__fadd2_rn(g[4], g[5]), __fadd2_rn(g[6], g[7]));
  return __fadd2_rn(__fadd2_rn(a, b), g[8]);
}
// keep = 1 - om for both nodes, a = om C_s per node, and minus w_i times the
// node's stored reference ((-w) r rounds to exactly -(w r))
struct PushK2 {
  float keep;
  float2 a, nwq[3];
};
__device__ __forceinline__ PushK2 push_k2(float om, float2 cs, float2 cqs) {
  PushK2 k;
  k.keep = __fsub_rn(1.0f, om);
  k.a = __fmul2_rn(dup(om), cs);
  k.nwq[0] = __fmul2_rn(dup(-w(0)), cqs);
  k.nwq[1] = __fmul2_rn(dup(-w(1)), cqs);
  k.nwq[2] = __fmul2_rn(dup(-w(5)), cqs);
  return k;
}
__device__ __forceinline__ float2 push2(int i, float2 g, float2 e, const PushK2 &k) {
  const float2 nwq = i == 0 ? k.nwq[0] : (i < 5 ? k.nwq[1] : k.nwq[2]);
  return __ffma2_rn(dup(k.keep), g, __ffma2_rn(k.a, e, nwq));
}

// Rounding of a scaled population to half.  LBM_F16_SR = 1 (default):
// stochastic rounding.  The float's 13 mantissa bits below half precision
// get a random 13-bit number added before truncation, so a value rounds up
// with probability equal to its distance from the lower neighbour and the
// rounding error has zero mean.  The random bits come from a hash of (node
// pair, step) times a per-store odd constant, so a run is reproducible.
// Round-to-nearest instead makes the iteration settle on a fixed point of
// the rounded map: near steady state the per-step change drops below half
// an ulp and the stored values stop moving.  On a 2048 x 512 cascade
// lattice that left the steady efficiency 2.5e-3 (3%) off the FP64 value;
// with stochastic rounding it is 2e-5 off, for 1.6% more step time.
#ifndef LBM_F16_SR
#define LBM_F16_SR 1
#endif
// LBM_PAIR_PER_SPECIES = 1 (default): the bulk pair kernel loads each
// species' 24 pairs just before that species' arithmetic, which needs 80
// registers (6 blocks per SM) instead of 122 (4 blocks) for all 72 pairs
// up front; with the L2 prefetch ahead the loads mostly hit L2, so the
// shorter load phases and 50% more resident warps win (1.634 ms per step
// of the 16384 x 4096 lattice against 1.692 ms).
#ifndef LBM_PAIR_PER_SPECIES
#define LBM_PAIR_PER_SPECIES 1
#endif
// Hash of (node pair, step) for the random bits.  Its constants are
// published integer-hash multipliers: 0x9E3779B1 (2^32 divided by the golden
// ratio, Knuth's multiplicative hashing), 0x85EBCA77 (the second 32-bit
// prime of xxHash), and the xor-shift-multiply finaliser with 0x7FEB352D,
// 0x846CA68B and shifts 16 / 15 / 16 (the "lowbias32" hash found by
// C. Wellons' hash prospector); 0x632BE5AB is an arbitrary odd offset.
__device__ __forceinline__ uint32_t pair_hash(long long pair, unsigned step) {
  uint32_t h = static_cast<uint32_t>(pair) * 0x9E3779B1u ^
               static_cast<uint32_t>(pair >> 32) * 0x7FEB352Du ^
               (step + 0x632BE5ABu) * 0x85EBCA77u;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return h;
}
// k: store index of the node pair (0 .. 2 * 27 - 1)
__device__ __forceinline__ __half round_half(float v, uint32_t h, int k) {
#if LBM_F16_SR
  const uint32_t r = (h * (0x9E3779B1u + 2u * static_cast<uint32_t>(k))) >> 19;
  return __float2half_rz(__uint_as_float(__float_as_uint(v) + r));
#else
  (void)h;
  (void)k;
  return __float2half_rn(v);
#endif
}
// The two nodes of a pair (lo: even x, hi: odd x) at store index k =
// 9 s + i.  LBM_F16_SR_HW = 1 (default): one cvt.rs instruction (this
// part's stochastic-rounding conversion) rounds both, with 32 random bits
// from the same hash; each half is rounded on its own, so the one-node form,
// which passes 0 for the other half, gets the same bits.  It measured 2.7%
// faster per step than round_half above (four instructions per value) with
// the same steady-state efficiency error.  LBM_F16_SR_HW = 0: round_half,
// element by element.
#ifndef LBM_F16_SR_HW
#define LBM_F16_SR_HW 1
#endif
__device__ __forceinline__ __half2 round_pair(float lo, float hi, uint32_t h,
                                              int k) {
#if LBM_F16_SR && LBM_F16_SR_HW
  const uint32_t r = h * (0x9E3779B1u + 2u * static_cast<uint32_t>(k));
  uint32_t d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
  __half2 out;
  memcpy(&out, &d, sizeof(d));
  return out;
#else
  return __halves2half2(round_half(lo, h, k), round_half(hi, h, 27 + k));
#endif
}
}  // namespace f16

template <int NS, int MODE>
__device__ __forceinline__ void adr_interior_node_f16(const AdrArgs &a, long long n,
                                                      float (&acc)[3 * NS]) {
  const long long np = a.nx_pad, plane = a.plane;
  const __half *__restrict__ src = static_cast<const __half *>(a.src);
  __half *__restrict__ dst = static_cast<__half *>(a.dst);
  const float *__restrict__ U = static_cast<const float *>(a.u);
  float g[NS][9];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const long long m = n - (cy(i) * np + cx(i));
      g[s][i] = f16::pull(i, __half2float(src[(long long)(s * 9 + i) * plane + m]),
                          __half2float(a.rsrc[s * plane + m]));
    }
  }
  float *__restrict__ cp = static_cast<float *>(a.cprev);
  float prev[NS];
  if (MODE == kAdrCheck) {
#pragma unroll
    for (int s = 0; s < NS; ++s) prev[s] = cp[s * plane + n];
  }
  float E[9];
  f16::eq(U[n], U[plane + n], E);
  const uint32_t h = f16::pair_hash(n >> 1, a.step);
  const bool odd = (n & 1) != 0;   // second node of its pair
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const float cs = f16::sum9(g[s]);
    const float c = __fmul_rn(cs, f16::kDown);
    const float cqs = __fmul_rn(ref_round(c), f16::kUp);
    a.rdst[s * plane + n] = __float2half_rn(c);
    const f16::PushK k = f16::push_k(a.fomega[s], cs, cqs);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      // rounded as one half of its pair, with the pair's random bits
      const float v = f16::push(i, g[s][i], E[i], k);
      const __half2 r2 = f16::round_pair(odd ? 0.0f : v, odd ? v : 0.0f, h,
                                         s * 9 + i);
      dst[(long long)(s * 9 + i) * plane + n] = odd ? __high2half(r2)
                                                    : __low2half(r2);
    }
    if (MODE == kAdrCheck) {
      check_add<NS, float>(acc, s, c, prev[s]);
      cp[s * plane + n] = c;
    }
  }
}

// FP16 bulk step, two nodes per thread: nodes (x0, x0 + 1), x0 even, of row
// y.  Every plane is read as aligned half2 pairs.  A pull with c_ix = +1
// takes the sources (x0 - 1, x0): the high half of the pair to the left and
// the low half of the node's own pair; c_ix = -1 takes (x0 + 1, x0 + 2)
// from the own pair and the pair to the right.  The left pair is needed only
// when node x0 is interior (its neighbour x0 - 1 is a lattice node, so
// x0 >= 2) and the right pair only when node x0 + 1 is interior (x0 + 2 <=
// nx - 1, so x0 + 3 < nx_pad): every read stays inside its row, and rows
// y +- 1 exist whenever either node is interior.  The reference
// concentrations of the source nodes come the same way (three rows of three
// pairs per species).  The arithmetic is that of adr_interior_node_f16.
// Launched with kBlockX / 2 threads on the grid of adr_bulk_kernel, so a
// block covers the same kBlockX nodes and writes the same partial-sum row.
//
// Each thread reads 24 pairs per species: slot 0..8 its own pair of plane
// i, 9..14 the side pair of the six planes with c_ix != 0 (directions 1, 3,
// 5, 6, 7, 8), 15..17 the centre reference pairs of rows y - 1, y, y + 1,
// 18..20 the left ones, 21..23 the right ones.
constexpr int kPairThreads = kBlockX / 2;
constexpr int kPairSlots = 24;
__device__ __forceinline__ constexpr int side_slot(int i) {
  return i == 1 ? 9 : i == 3 ? 10 : i == 5 ? 11 : i == 6 ? 12 : i == 7 ? 13 : 14;
}
// global address of slot k of species s for the pair at (y, x0), and
// whether the pair is needed (side pairs only for an interior neighbour)
struct PairSrc {
  const __half *p;
  bool need;
};
__device__ __forceinline__ PairSrc pair_src(const AdrArgs &a, int s, int k,
                                            int y, int x0, bool in0, bool in1) {
  const long long np = a.nx_pad, plane = a.plane;
  const __half *src = static_cast<const __half *>(a.src);
  if (k < 9) {
    return {src + (long long)(s * 9 + k) * plane + (long long)(y - cy(k)) * np + x0,
            true};
  }
  if (k < 15) {
    const int i = k == 9 ? 1 : k == 10 ? 3 : k == 11 ? 5 : k == 12 ? 6 : k == 13 ? 7 : 8;
    const __half *row = src + (long long)(s * 9 + i) * plane + (long long)(y - cy(i)) * np + x0;
    return cx(i) > 0 ? PairSrc{row - 2, in0} : PairSrc{row + 2, in1};
  }
  const int r = (k - 15) % 3, side = (k - 15) / 3;   // 0 centre, 1 left, 2 right
  const __half *row = a.rsrc + (long long)s * plane + (long long)(y + r - 1) * np + x0;
  return side == 0 ? PairSrc{row, true} : side == 1 ? PairSrc{row - 2, in0}
                                                   : PairSrc{row + 2, in1};
}

// The update of the pair from its 24 x NS source pairs, fetched by
// fetch(s, k) (k as above; a side pair that is not needed may hold
// anything).  Stores the new populations, references and, on check steps,
// the recorded concentrations, and adds the check-step values to acc.
template <int NS, int MODE, class Fetch>
__device__ __forceinline__ void pair_update(const AdrArgs &a, int y, int x0,
                                            bool in0, bool in1, float2 ux,
                                            float2 uy, Fetch &&fetch,
                                            float (&acc)[2][3 * NS]) {
  const long long np = a.nx_pad, plane = a.plane;
  const long long n0 = (long long)y * np + x0;
  __half *__restrict__ dst = static_cast<__half *>(a.dst);
  float *__restrict__ cp = static_cast<float *>(a.cprev);
  float2 prev[NS];
  if (MODE == kAdrCheck) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
      prev[s] = *reinterpret_cast<const float2 *>(cp + s * plane + n0);
  }
  float2 E[9];
  f16::eq2(ux, uy, E);
  const uint32_t hp = f16::pair_hash(n0 >> 1, a.step);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    // references of the source columns x0 - 1 .. x0 + 2, rows
    // y - 1 .. y + 1 (the left / right column only where it is read)
    float rs[3][4];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float2 c2 = __half22float2(fetch(s, 15 + r));
      rs[r][0] = __high2float(fetch(s, 18 + r));
      rs[r][1] = c2.x;
      rs[r][2] = c2.y;
      rs[r][3] = __low2float(fetch(s, 21 + r));
    }
    float2 g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int r = 1 - cy(i);      // source row y - cy(i)
      const int k = 1 - cx(i);      // column of node x0's source, x0 - 1 + k
      const __half2 own = fetch(s, i);
      __half2 h;
      if (cx(i) == 0) h = own;
      else if (cx(i) > 0) h = __halves2half2(__high2half(fetch(s, side_slot(i))), __low2half(own));
      else h = __halves2half2(__high2half(own), __low2half(fetch(s, side_slot(i))));
      g[i] = __ffma2_rn(f16::dup(f16::w(i) * f16::kUp),
                        make_float2(rs[r][k], rs[r][k + 1]), __half22float2(h));
    }
    const float2 cs = f16::sum9(g);
    const float2 c = __fmul2_rn(cs, f16::dup(f16::kDown));
    const __half2 cr = __float22half2_rn(c);   // the stored references
    const float2 cq = __fmul2_rn(__half22float2(cr), f16::dup(f16::kUp));
    const f16::PushK2 kk = f16::push_k2(a.fomega[s], cs, cq);
    __half *o = dst + (long long)s * 9 * plane + n0;
    __half *ro = a.rdst + (long long)s * plane + n0;
    float *co = cp + s * plane + n0;
    if (in0 && in1) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const float2 v = f16::push2(i, g[i], E[i], kk);
        *reinterpret_cast<__half2 *>(o + (long long)i * plane) =
            f16::round_pair(v.x, v.y, hp, s * 9 + i);
      }
      *reinterpret_cast<__half2 *>(ro) = cr;
      if (MODE == kAdrCheck) *reinterpret_cast<float2 *>(co) = c;
    } else {
      // one interior node: the other belongs to the boundary kernel
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const float2 v = f16::push2(i, g[i], E[i], kk);
        const __half2 r2 = f16::round_pair(in0 ? v.x : 0.0f, in1 ? v.y : 0.0f, hp,
                                           s * 9 + i);
        if (in0) o[(long long)i * plane] = __low2half(r2);
        if (in1) o[(long long)i * plane + 1] = __high2half(r2);
      }
      if (in0) ro[0] = __low2half(cr);
      if (in1) ro[1] = __high2half(cr);
      if (MODE == kAdrCheck) {
        if (in0) co[0] = c.x;
        if (in1) co[1] = c.y;
      }
    }
    if (MODE == kAdrCheck) {
      if (in0) check_add<NS, float>(acc[0], s, c.x, prev[s].x);
      if (in1) check_add<NS, float>(acc[1], s, c.y, prev[s].y);
    }
  }
}

// The bulk kernel.  A block first sends the L2 prefetches for the block
// LBM_PREFETCH_ROWS_F16 rows below it, then each thread loads its pairs
// (per species by default, or all 24 x NS before any arithmetic with
// LBM_PAIR_PER_SPECIES = 0) and updates its two nodes.  The check-step form
// keeps its partial sums as well and is bounded at 5 blocks per SM (96
// registers) so that it does not spill.
template <int NS, int MODE>
__global__ void __launch_bounds__(kPairThreads, MODE == kAdrCheck ? 5 : LBM_PAIR_MIN_BLOCKS)
    adr_bulk_pair_kernel(const AdrArgs a) {
  const int y = blockIdx.y;
  if (LBM_PREFETCH_ROWS_F16 > 0)
    bulk_prefetch_rows<__half, float, NS, true>(a, y + LBM_PREFETCH_ROWS_F16);
  const int x0 = 2 * (blockIdx.x * kPairThreads + threadIdx.x);
  const long long n0 = (long long)y * a.nx_pad + x0;
  uint2 lw = make_uint2(kSolidNode, kSolidNode);
  if (x0 < a.nx_pad) lw = *reinterpret_cast<const uint2 *>(a.links + n0);
  const bool in0 = lw.x == 0u, in1 = lw.y == 0u;
  float acc[2][3 * NS];   // check-step values of node x0 and of node x0 + 1
#pragma unroll
  for (int k = 0; k < 3 * NS; ++k) acc[0][k] = acc[1][k] = 0.0f;
  if (in0 || in1) {
    const __half2 z2 = __float2half2_rn(0.0f);
    const float *__restrict__ U = static_cast<const float *>(a.u);
    const float2 ux = *reinterpret_cast<const float2 *>(U + n0);
    const float2 uy = *reinterpret_cast<const float2 *>(U + a.plane + n0);
#if LBM_PAIR_PER_SPECIES
    // each species' pairs are loaded as its arithmetic needs them (the
    // stores of one species keep the next one's loads behind them)
    pair_update<NS, MODE>(a, y, x0, in0, in1, ux, uy, [&](int s, int k) {
      const PairSrc q = pair_src(a, s, k, y, x0, in0, in1);
      return q.need ? *reinterpret_cast<const __half2 *>(q.p) : z2;
    }, acc);
#else
    __half2 v[NS][kPairSlots];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
      for (int k = 0; k < kPairSlots; ++k) {
        const PairSrc q = pair_src(a, s, k, y, x0, in0, in1);
        v[s][k] = q.need ? *reinterpret_cast<const __half2 *>(q.p) : z2;
      }
    }
    pair_update<NS, MODE>(a, y, x0, in0, in1, ux, uy,
                          [&](int s, int k) { return v[s][k]; }, acc);
#endif
  }
  if constexpr (MODE == kAdrCheck) {
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    block_partials_store<2 * NS, NS, 2, kPairThreads, float>(
        acc, a.partials + b * (3 * NS));
  }
}

// FP16 plain step, four nodes per thread: nodes x0 .. x0 + 3 (x0 a multiple
// of 4) of row y, with every plane read and written as aligned 8-byte
// quads.  A pull with c_ix = +1 takes the sources x0 - 1 .. x0 + 2: the
// last half of the quad to the left (one 2-byte load) and three halves of
// the node's own quad; c_ix = -1 takes x0 + 1 .. x0 + 4, the first half of
// the quad to the right.  The left half is loaded only when node x0 is
// interior (then x0 - 1 is a lattice node) and the right one only when node
// x0 + 3 is (then x0 + 4 <= nx - 1 < nx_pad); rows y +- 1 exist whenever a
// node of the quad is interior.  The reference concentrations come the same
// way, three rows of one quad and two single halves per species.  Against
// the two-node kernel this halves the load instructions and the address
// arithmetic per node.  The arithmetic is that of pair_update on the pairs
// (x0, x0 + 1) and (x0 + 2, x0 + 3), operation for operation (the same
// packed roundings, the same random bits per pair), so every stored half is
// the two-node kernel's.  Plain steps only: check steps keep the two-node
// kernel, which also writes the partial sums.  Launched with kBlockX / 4
// threads on the grid of adr_bulk_kernel.
#ifndef LBM_QUAD_MIN_BLOCKS
#define LBM_QUAD_MIN_BLOCKS 8
#endif
constexpr int kQuadThreads = kBlockX / 4;

template <int NS>
__global__ void __launch_bounds__(kQuadThreads, LBM_QUAD_MIN_BLOCKS)
    adr_bulk_quad_kernel(const AdrArgs a) {
  static_assert(kQuadThreads >= 9 * NS + NS + 3, "one prefetch per thread");
  static_assert(kQuadThreads % 32 == 0, "whole warps");
  const int y = blockIdx.y;
  if (LBM_PREFETCH_ROWS_F16 > 0)
    bulk_prefetch_rows<__half, float, NS, true>(a, y + LBM_PREFETCH_ROWS_F16);
  const int x0 = 4 * (blockIdx.x * kQuadThreads + threadIdx.x);
  if (x0 >= a.nx_pad) return;   // nx_pad is a multiple of 4: x0 + 3 < nx_pad
  const long long np = a.nx_pad, plane = a.plane;
  const long long n0 = (long long)y * np + x0;
  const uint4 lw = *reinterpret_cast<const uint4 *>(a.links + n0);
  const bool in0 = lw.x == 0u, in1 = lw.y == 0u, in2 = lw.z == 0u, in3 = lw.w == 0u;
  if (!(in0 || in1 || in2 || in3)) return;
  const bool all = in0 && in1 && in2 && in3;
  const __half *src = static_cast<const __half *>(a.src);
  __half *__restrict__ dst = static_cast<__half *>(a.dst);
  const float *__restrict__ U = static_cast<const float *>(a.u);
  const float4 ux = *reinterpret_cast<const float4 *>(U + n0);
  const float4 uy = *reinterpret_cast<const float4 *>(U + plane + n0);
  float2 El[9], Eh[9];
  f16::eq2(make_float2(ux.x, ux.y), make_float2(uy.x, uy.y), El);
  f16::eq2(make_float2(ux.z, ux.w), make_float2(uy.z, uy.w), Eh);
  // random bits of the pairs (x0, x0 + 1) and (x0 + 2, x0 + 3)
  const uint32_t hl = f16::pair_hash(n0 >> 1, a.step);
  const uint32_t hh = f16::pair_hash((n0 >> 1) + 1, a.step);
  const __half hz = __float2half_rn(0.0f);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    // the species' loads, issued before its arithmetic: nine own quads,
    // six side halves, and per row y - 1 .. y + 1 the reference quad with
    // its two side halves
    uint2 q[9];
    __half side[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const __half *row = src + (long long)(s * 9 + i) * plane +
                          (long long)(y - cy(i)) * np + x0;
      q[i] = *reinterpret_cast<const uint2 *>(row);
      side[i] = hz;
      if (cx(i) > 0 && in0) side[i] = row[-1];
      if (cx(i) < 0 && in3) side[i] = row[4];
    }
    uint2 rq[3];
    __half rl[3], rr[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const __half *row = a.rsrc + (long long)s * plane + (long long)(y + r - 1) * np + x0;
      rq[r] = *reinterpret_cast<const uint2 *>(row);
      rl[r] = in0 ? row[-1] : hz;
      rr[r] = in3 ? row[4] : hz;
    }
    // reference concentrations of the source columns x0 - 1 .. x0 + 4
    float rs[3][6];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      __half2 lo, hi;
      memcpy(&lo, &rq[r].x, 4);
      memcpy(&hi, &rq[r].y, 4);
      const float2 fl = __half22float2(lo), fh = __half22float2(hi);
      rs[r][0] = __half2float(rl[r]);
      rs[r][1] = fl.x;
      rs[r][2] = fl.y;
      rs[r][3] = fh.x;
      rs[r][4] = fh.y;
      rs[r][5] = __half2float(rr[r]);
    }
    float2 gl[9], gh[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int r = 1 - cy(i);   // source row y - cy(i)
      const int k = 1 - cx(i);   // column of node x0's source, x0 - 1 + k
      __half2 lo, hi;
      memcpy(&lo, &q[i].x, 4);
      memcpy(&hi, &q[i].y, 4);
      const float2 fl = __half22float2(lo), fh = __half22float2(hi);
      const float p[6] = {__half2float(side[i]), fl.x, fl.y, fh.x, fh.y,
                          __half2float(side[i])};
      const float2 wk = f16::dup(f16::w(i) * f16::kUp);
      gl[i] = __ffma2_rn(wk, make_float2(rs[r][k], rs[r][k + 1]),
                         make_float2(p[k], p[k + 1]));
      gh[i] = __ffma2_rn(wk, make_float2(rs[r][k + 2], rs[r][k + 3]),
                         make_float2(p[k + 2], p[k + 3]));
    }
    const float2 csl = f16::sum9(gl), csh = f16::sum9(gh);
    const float2 cl = __fmul2_rn(csl, f16::dup(f16::kDown));
    const float2 ch = __fmul2_rn(csh, f16::dup(f16::kDown));
    const __half2 crl = __float22half2_rn(cl), crh = __float22half2_rn(ch);
    const f16::PushK2 kl = f16::push_k2(
        a.fomega[s], csl, __fmul2_rn(__half22float2(crl), f16::dup(f16::kUp)));
    const f16::PushK2 kh = f16::push_k2(
        a.fomega[s], csh, __fmul2_rn(__half22float2(crh), f16::dup(f16::kUp)));
    __half *o = dst + (long long)s * 9 * plane + n0;
    __half *ro = a.rdst + (long long)s * plane + n0;
    if (all) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const float2 vl = f16::push2(i, gl[i], El[i], kl);
        const float2 vh = f16::push2(i, gh[i], Eh[i], kh);
        const __half2 rl2 = f16::round_pair(vl.x, vl.y, hl, s * 9 + i);
        const __half2 rh2 = f16::round_pair(vh.x, vh.y, hh, s * 9 + i);
        uint2 w;
        memcpy(&w.x, &rl2, 4);
        memcpy(&w.y, &rh2, 4);
        *reinterpret_cast<uint2 *>(o + (long long)i * plane) = w;
      }
      uint2 w;
      memcpy(&w.x, &crl, 4);
      memcpy(&w.y, &crh, 4);
      *reinterpret_cast<uint2 *>(ro) = w;
    } else {
      // some nodes of the quad belong to the boundary kernel (or are
      // solid): store the interior ones, each rounded as in the two-node
      // kernel with zero in the lane of a node it does not store
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const float2 vl = f16::push2(i, gl[i], El[i], kl);
        const float2 vh = f16::push2(i, gh[i], Eh[i], kh);
        const __half2 rl2 = f16::round_pair(in0 ? vl.x : 0.0f, in1 ? vl.y : 0.0f,
                                            hl, s * 9 + i);
        const __half2 rh2 = f16::round_pair(in2 ? vh.x : 0.0f, in3 ? vh.y : 0.0f,
                                            hh, s * 9 + i);
        __half *oi = o + (long long)i * plane;
        if (in0) oi[0] = __low2half(rl2);
        if (in1) oi[1] = __high2half(rl2);
        if (in2) oi[2] = __low2half(rh2);
        if (in3) oi[3] = __high2half(rh2);
      }
      if (in0) ro[0] = __low2half(crl);
      if (in1) ro[1] = __high2half(crl);
      if (in2) ro[2] = __low2half(crh);
      if (in3) ro[3] = __high2half(crh);
    }
  }
}

}  // namespace lbm
