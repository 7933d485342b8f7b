// Tensor-core Gram sweep (paper Section 4 'gram'; batches of Section 3.1) with TF32 or BF16
// operands and FP32 accumulation in tensor memory (tcgen05).
//
// A CTA owns a tile of TA x TB pairs (a, b) with TA = 128 / RA and TB = 128 / RB, RA and RB the
// ranks of the two sides zero-padded to 16, 32 or 64. Per mode slice i of core k the
// left-partial update M'_ab = sum_i A_a,i^T M_ab B_b,i is two tensor-core products with M = 128:
//   MMA1 (one per b)  T[(a,al), bp]   = sum_be M_b[(a,al), be] B_b,i[be, bp]   TMEM columns b*RB + bp
//   MMA2 (one per a)  D_a[(b,bp), ap] += sum_al T_a[(b,bp), al] A_a,i[al, ap]  TMEM columns 128 + a*RA + ap
// T goes TMEM -> registers -> shared memory (rounded to the operand type) between the two
// products; D accumulates the n_k slices of core k in FP32 and becomes the next core's M the
// same way. The final M_d (1 x 1 per pair) is <A_a, B_b>.
//
// Shared-memory operands are K-major without swizzle: 8-row x 16-byte core matrices, rows 16
// bytes apart, core matrices 144 bytes apart along K (a 16-byte skew, so that the column
// writes of the epilogues fall on distinct banks) and SBO = (K / elements-per-16-bytes) * 144
// bytes apart along M/N. Padded rows and columns hold exact zeros, so padding never changes a
// result.
#include <algorithm>
#include <string.h>

#include "gram_mma.cuh"

namespace t3f {

namespace {

constexpr int kMmaThreads = 256;
constexpr uint32_t kTmemCols = 256;  // T at columns 0..127, D at 128..255
constexpr uint32_t kTmemColsPipe = 512;  // pipelined: a second T at columns 256..383
constexpr uint32_t kSkew = 64;  // extra bytes between consecutive operands (16-bank shift)

constexpr uint32_t kSmemCap = 227u * 1024u;

// Shared-memory plan of a tile shape (RA, RB) for element size es: operand strides, region
// offsets, and whether the slice operands fit twice (double buffering).
struct MmaLayout {
  uint32_t sbo_a, sbo_b, big_a, big_b, sl_a, sl_b;  // SBO and operand strides (bytes)
  uint32_t o_as, o_mop, o_top, total;
  int nbuf;
};

__host__ __device__ constexpr MmaLayout mma_layout(int es, int RA, int RB) {
  MmaLayout L{};
  const uint32_t T = 16u / (uint32_t)es;
  L.sbo_a = (uint32_t)RA / T * kLBO;
  L.sbo_b = (uint32_t)RB / T * kLBO;
  L.big_a = 16u * L.sbo_a + kSkew;               // T_a: 128 rows, K = RA
  L.big_b = 16u * L.sbo_b + kSkew;               // M_b: 128 rows, K = RB
  L.sl_a = (uint32_t)RA / 8u * L.sbo_a + kSkew;  // A_a,i: RA rows, K = RA
  L.sl_b = (uint32_t)RB / 8u * L.sbo_b + kSkew;  // B_b,i: RB rows, K = RB
  const uint32_t TA = 128u / (uint32_t)RA, TB = 128u / (uint32_t)RB;
  const uint32_t slices = TB * L.sl_b + TA * L.sl_a, bigs = TB * L.big_b + TA * L.big_a;
  L.nbuf = 2u * slices + bigs <= kSmemCap ? 2 : 1;
  // regions: B slices [nbuf][TB], A slices [nbuf][TA], M_b [TB], T_a [TA]
  L.o_as = (uint32_t)L.nbuf * TB * L.sl_b;
  L.o_mop = L.o_as + (uint32_t)L.nbuf * TA * L.sl_a;
  L.o_top = L.o_mop + TB * L.big_b;
  L.total = L.o_top + TA * L.big_a;
  return L;
}

// Pipelined variant (BF16 work lists): three slice buffers and two copies of T_a, so that
// slice i + 1's first product runs while slice i's T is transposed.
__host__ __device__ constexpr MmaLayout mma_layout_pipe(int es, int RA, int RB) {
  MmaLayout L = mma_layout(es, RA, RB);
  const uint32_t TA = 128u / (uint32_t)RA, TB = 128u / (uint32_t)RB;
  L.nbuf = 3;
  L.o_as = 3u * TB * L.sl_b;
  L.o_mop = L.o_as + 3u * TA * L.sl_a;
  L.o_top = L.o_mop + TB * L.big_b;
  L.total = L.o_top + 2u * TA * L.big_a;
  return L;
}

struct GramMmaArgs {
  TTV A, B;                   // uniform mode: the two batches (A the side of the smaller rank)
  float* out;                 // uniform mode: out[a * ldo + b], or out[b * ldo + a] if swap
  int ldo, swap;
  int* err;                   // device error word (nullable)
  uint32_t smem_bytes;
  int mode;                   // 0: tile from blockIdx (uniform), 1: persistent work list (groups)
  // work-list mode: ragged objects in rank-sorted positions
  const void* cores;
  const long long* off;       // [pos][dmax] element offset of core k
  const int* rk;              // [pos][dmax + 1] ranks
  int dmax;
  const int* nmodes;          // [group][dmax]
  const int* gd;              // [group] d
  const int* gstart;          // [group + 1]
  const int* perm;            // [pos] index of the object within its group
  const long long* gout_off;  // [group] offset of the group's S x S matrix in gout
  float* gout;
  const int* items;           // [item][8]: group, a0, na, b0, nb, RA, sym, RB
  int nitems;
  int* head;                  // work-list counter
  // adjoint sweeps (k_gram_mma_sweeps): the partials of every interface go to scratch slots
  char* scr;                  // scratch base
  const long long* soff;      // work-list mode: first slot orientation of item w (128 x 128 operands)
  long long sstride;          // uniform mode: slot orientations of one tile
  const float* gcot;          // cotangent: work list [group][S][S] (gout_off, perm); uniform dG
  int ldg;                    // uniform: row stride of dG
};

// BF16 transposing epilogue: TMEM rows (x, kappa) (x = row / RL) and columns m = 0..127 go to
// operand x at (row m, K = kappa) of a K-major BF16 operand array (operand stride BIG, row
// groups SBO apart). Each warp covers the 32 lanes of its quarter and 64 of the columns; every
// 16 x 16 block is two TMEM loads, four packs and one transposing matrix store.
template <int RL, uint32_t SBO, uint32_t BIG>
__device__ __forceinline__ void epi_bf16(uint32_t tcol, char* dst) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, h = warp >> 2;
  const int mi = lane >> 3, j = lane & 7;
#pragma unroll
  for (int win = 0; win < 2; ++win) {
    const int L0 = q * 32 + win * 16;
    const int x = L0 / RL, k0 = L0 % RL;
    uint32_t r[4][8];
#pragma unroll
    for (int cb = 0; cb < 4; ++cb) tmem_ld_16x16(tcol + ((uint32_t)L0 << 16) + (uint32_t)(h * 64 + cb * 16), r[cb]);
    tmem_wait_ld();
    char* base = dst + x * BIG + (uint32_t)(k0 / 8 + (mi & 1)) * kLBO + (uint32_t)j * 16u;
#pragma unroll
    for (int cb = 0; cb < 4; ++cb) {
      const int col = h * 64 + cb * 16 + (mi >> 1) * 8;  // this lane's matrix column block
      const uint32_t addr = su32(base + (uint32_t)(col >> 3) * SBO);
      asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1,%2,%3,%4};" ::"r"(addr),
                   "r"(bf2(r[cb][0], r[cb][1])), "r"(bf2(r[cb][2], r[cb][3])), "r"(bf2(r[cb][4], r[cb][5])),
                   "r"(bf2(r[cb][6], r[cb][7]))
                   : "memory");
    }
  }
}

// Same transposition element by element (any operand type): thread = TMEM row.
template <int KIND, int RL, uint32_t SBO, uint32_t BIG>
__device__ __forceinline__ void epi_scalar(uint32_t tcol, char* dst) {
  using O = OpT<KIND>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, h = warp >> 2;
  const int row = q * 32 + lane, x = row / RL, kk = row % RL;
  char* d = dst + x * BIG;
#pragma unroll
  for (int cc = 0; cc < 64; cc += 16) {
    const int c0 = h * 64 + cc;
    float v[16];
    tmem_ld16(tcol + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) O::st(d + eoff<O::ES>(c0 + jj, kk, SBO), v[jj]);
  }
}

template <int KIND, int RL, uint32_t SBO, uint32_t BIG>
__device__ __forceinline__ void epi_transpose(uint32_t tcol, char* dst) {
  if constexpr (KIND == 1)
    epi_bf16<RL, SBO, BIG>(tcol, dst);
  else
    epi_scalar<KIND, RL, SBO, BIG>(tcol, dst);
}

// Everything a CTA keeps across the tiles it processes.
struct MmaState {
  uint32_t tmem, bar1, bar2, ph1, ph2;
  bool pending1, pending2;  // a committed product batch not yet waited for
  // pipelined loop: one barrier per T buffer (first products) and per T copy (second
  // products), so that no barrier ever has two completions outstanding
  uint32_t b1[2], b2[2], q1[2], q2[2];  // indexed by constants or through the pipe_* helpers
  bool pd1[2], pd2[2];
  uint32_t cols;            // tensor-memory columns allocated
  int bad;                  // this thread saw a wait run out
  long long* s_base;        // [2 core parities][2 sides][8 objects]
  int* s_r0;                // K (left-rank) limit of the swept core
  int* s_r1;                // row (right-rank) limit
  int* s_cs;                // element strides of the slice operand: K index, row index, mode index
  int* s_rs;
  int* s_is;
  float* s_g;               // adjoint sweeps: cotangent of pair (a, b) at [a * 8 + b]
};


// Pipelined loop helpers: wait for / record a product batch on barrier pair `which` (1: first
// products, 2: second products), buffer p; p selects between scalars so nothing is indexed at
// run time (which would move the state to local memory).
__device__ __forceinline__ void pipe_wait(MmaState& st, int which, int p) {
  uint32_t& ph = which == 1 ? (p ? st.q1[1] : st.q1[0]) : (p ? st.q2[1] : st.q2[0]);
  bool& pd = which == 1 ? (p ? st.pd1[1] : st.pd1[0]) : (p ? st.pd2[1] : st.pd2[0]);
  const uint32_t bar = which == 1 ? (p ? st.b1[1] : st.b1[0]) : (p ? st.b2[1] : st.b2[0]);
  if (pd) {
    st.bad |= !mbar_wait(bar, ph);
    ph ^= 1u;
    pd = false;
  }
}
__device__ __forceinline__ void pipe_commit(MmaState& st, int which, int p) {
  const uint32_t bar = which == 1 ? (p ? st.b1[1] : st.b1[0]) : (p ? st.b2[1] : st.b2[0]);
  if (threadIdx.x == 0) mma_commit(bar);
}
__device__ __forceinline__ void pipe_mark(MmaState& st, int which, int p) {
  bool& pd = which == 1 ? (p ? st.pd1[1] : st.pd1[0]) : (p ? st.pd2[1] : st.pd2[0]);
  pd = true;
}

// Adjoint sweeps: the partial D (TMEM columns from tcol; lanes (b, be), columns (a, al)) goes
// to one scratch slot in two orientations, each a 128 x 128 K-major operand with 16-byte core
// matrices packed along K (LBO 128 bytes, SBO 16 * 128 bytes per 8 rows):
//   o1: rows (b, be), K = (a, al)          o0: rows (a, al), K = (b, be)
// rounded to the operand type and scaled by the pair's cotangent when sg is given.
template <int KIND, int RA, int RB>
__device__ __forceinline__ void store_partial(uint32_t tcol, char* o0, char* o1, const float* sg) {
  using O = OpT<KIND>;
  constexpr int ES = O::ES, T = 16 / ES;
  constexpr uint32_t SBO = (128u / T) * 128u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, h = warp >> 2;
  const int row = q * 32 + lane, b = row / RB;
#pragma unroll
  for (int cc = 0; cc < 64; cc += 16) {
    const int c0 = h * 64 + cc;
    float v[16];
    tmem_ld16(tcol + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
    if (sg) {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] *= sg[((c0 + j) / RA) * 8 + b];
    }
#pragma unroll
    for (int ch = 0; ch < 16 / T; ++ch) {
      float u[T];
#pragma unroll
      for (int t = 0; t < T; ++t) u[t] = v[ch * T + t];
      *reinterpret_cast<uint4*>(o1 + (uint32_t)(row >> 3) * SBO + (uint32_t)((c0 + ch * T) / T) * 128u +
                                (uint32_t)(row & 7) * 16u) = O::pack(u);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int c = c0 + j;
      O::st(o0 + (uint32_t)(c >> 3) * SBO + (uint32_t)(row / T) * 128u + (uint32_t)(c & 7) * 16u +
                (uint32_t)(row % T) * ES,
            v[j]);
    }
  }
}

// One tile: na x nb pairs (a0.., b0..) of one group (or of the uniform batches), d cores.
// Returns false (block-uniformly) when a tensor-core wait ran out.
// Adjoint sweeps (slots != nullptr): dir 0 runs the left sweep and stores M_0 .. M_{d-1};
// dir 1 runs the same recursion over the cores in reverse order with transposed slices
// (R_k = sum_i A_k,i R_{k+1} B_k,i^T) and stores R_1 .. R_d. Slot j of direction dir holds
// interface j (dir 0) or j + 1 (dir 1); M is stored scaled by the pair's cotangent.
// PIPE (BF16 work lists): three slice buffers, T and its shared-memory copy double-buffered;
// slice i + 1's first product is issued before slice i's T is transposed.
template <int KIND, int RA, int RB, typename ST, bool PIPE = false>
__device__ bool mma_tile_sync(const GramMmaArgs& g, char* sm, MmaState& st, int grp, int a0, int na, int b0, int nb,
                              int sym, int d, int dir = 0, char* slots = nullptr) {
  using O = OpT<KIND>;
  constexpr int ES = O::ES;
  constexpr int T = 16 / ES;
  constexpr int TA = 128 / RA, TB = 128 / RB;
  constexpr MmaLayout L = PIPE ? mma_layout_pipe(ES, RA, RB) : mma_layout(ES, RA, RB);
  constexpr int NBUF = L.nbuf;
  constexpr uint32_t SBOA = L.sbo_a, SBOB = L.sbo_b, BIGA = L.big_a, BIGB = L.big_b, SLA = L.sl_a, SLB = L.sl_b;
  constexpr uint32_t ID1 = idesc(O::FMT, RB), ID2 = idesc(O::FMT, RA);
  constexpr int KGA = RA / T, KGB = RB / T;                        // K groups of T elements
  constexpr int UPA = TA * RA * KGA / kMmaThreads, UPB = TB * RB * KGB / kMmaThreads;
  constexpr int USA = kMmaThreads / RA, USB = kMmaThreads / RB;
  static_assert(UPA * kMmaThreads == TA * RA * KGA && UPB * kMmaThreads == TB * RB * KGB, "staging split");
  static_assert(L.total <= kSmemCap, "tile does not fit");

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  char* const bsl = sm;
  char* const asl = sm + L.o_as;
  char* const mop = sm + L.o_mop;
  char* const top = sm + L.o_top;
  const void* const Ap = g.mode == 0 ? g.A.p : g.cores;
  const void* const Bp = g.mode == 0 ? g.B.p : g.cores;
  const int q = warp & 3, h = warp >> 2;   // TMEM lane quarter, column half
  const int row = q * 32 + lane;           // TMEM lane = operand row of this thread
  const int srA = tid % RA, suA = tid / RA, srB = tid % RB, suB = tid / RB;
  long long(*s_base)[2][8] = reinterpret_cast<long long(*)[2][8]>(st.s_base);
  int(*s_r0)[2][8] = reinterpret_cast<int(*)[2][8]>(st.s_r0);
  int(*s_r1)[2][8] = reinterpret_cast<int(*)[2][8]>(st.s_r1);
  int(*s_cs)[2][8] = reinterpret_cast<int(*)[2][8]>(st.s_cs);
  int(*s_rs)[2][8] = reinterpret_cast<int(*)[2][8]>(st.s_rs);
  int(*s_is)[2][8] = reinterpret_cast<int(*)[2][8]>(st.s_is);
  constexpr uint32_t kSlot = 128u * 128u * ES;  // bytes of one orientation of a slot

  // swept core k is stored core kc (reversed for dir 1)
  auto nmode = [&](int k) {
    const int kc = dir ? d - 1 - k : k;
    return g.mode == 0 ? g.A.n[kc] : g.nmodes[grp * g.dmax + kc];
  };
  // per-object core offsets and ranks of core k into parity slot par (missing objects: rank 0)
  // (the slice operand's rows are the swept core's right-rank index, K its left-rank index;
  // reversed, the stored core's left and right ranks trade places)
  auto fill_info = [&](int k, int par) {
    if (tid < 16) {
      const int side = tid / 8, o = tid % 8, cnt = side ? nb : na, o0 = side ? b0 : a0;
      const int kc = dir ? d - 1 - k : k;
      long long base = 0;
      int rl = 0, rr = 0;
      if (o < cnt) {
        if (g.mode == 0) {
          const TTV& V = side ? g.B : g.A;
          base = V.off[kc] + (long long)(o0 + o) * V.osz[kc];
          rl = V.r[kc];
          rr = V.r[kc + 1];
        } else {
          const int pos = o0 + o;
          base = g.off[(long long)pos * g.dmax + kc];
          rl = g.rk[(long long)pos * (g.dmax + 1) + kc];
          rr = g.rk[(long long)pos * (g.dmax + 1) + kc + 1];
        }
      }
      const int n = nmode(k), row_stride = n * rr;
      s_base[par][side][o] = base;
      s_r0[par][side][o] = dir ? rr : rl;
      s_r1[par][side][o] = dir ? rl : rr;
      s_cs[par][side][o] = dir ? 1 : row_stride;
      s_rs[par][side][o] = dir ? row_stride : 1;
      s_is[par][side][o] = rr;
    }
  };
  // M_0 = 1 for every pair: zero all M_b, then element (row a*RA, col 0) of every M_b
  for (uint32_t e = (uint32_t)tid * 16u; e < TB * BIGB; e += kMmaThreads * 16u)
    *reinterpret_cast<uint4*>(mop + e) = make_uint4(0u, 0u, 0u, 0u);
  fill_info(0, 0);
  if (slots) {
    // the pairs' cotangents, and the boundary slot: M_0 (scaled) or R_d, one at (a*RA, b*RB)
    if (tid < 64) {
      const int a = tid / 8, b = tid % 8;
      float gv = 0.f;
      if (a < na && b < nb) {
        if (g.mode == 0) {
          gv = g.swap ? g.gcot[(long long)(b0 + b) * g.ldg + (a0 + a)] : g.gcot[(long long)(a0 + a) * g.ldg + (b0 + b)];
        } else {
          const long long S = g.gstart[grp + 1] - g.gstart[grp];
          const long long la = g.perm[a0 + a], lb = g.perm[b0 + b];
          const float* o = g.gcot + g.gout_off[grp];
          gv = o[la * S + lb] + (sym ? o[lb * S + la] : 0.f);
        }
      }
      st.s_g[tid] = gv;
    }
    char* const o0 = slots + (size_t)((dir * d + (dir ? d - 1 : 0)) * 2) * kSlot;
    for (uint32_t e = (uint32_t)tid * 16u; e < 2u * kSlot; e += kMmaThreads * 16u)
      *reinterpret_cast<uint4*>(o0 + e) = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (tid < TA * TB) {
      constexpr uint32_t SB = (128u / T) * 128u;
      const int a = tid / TB, b = tid % TB, ra = a * RA, rb = b * RB;
      const float v = (a < na && b < nb) ? (dir ? 1.f : st.s_g[a * 8 + b]) : 0.f;
      O::st(o0 + (uint32_t)(ra >> 3) * SB + (uint32_t)(rb / T) * 128u + (uint32_t)(ra & 7) * 16u, v);
      O::st(o0 + kSlot + (uint32_t)(rb >> 3) * SB + (uint32_t)(ra / T) * 128u + (uint32_t)(rb & 7) * 16u, v);
    }
  }
  __syncthreads();
  if (tid < TA * TB) O::st(mop + (tid / TA) * BIGB + eoff<ES>((tid % TA) * RA, 0, SBOB), 1.0f);

  // slice i of core k of both sides -> registers. K run j of this thread on side X covers
  // object o = (suX + j*USX) / KGX, columns c = ((suX + j*USX) % KGX) * T + t, row srX
  uint32_t pb[UPB][T], pa[UPA][T];
  auto load_slice = [&](int k, int i) {
    const int par = k & 1;
#pragma unroll
    for (int j = 0; j < UPB; ++j) {
      const int w = suB + j * USB, o = w / KGB, c0 = (w % KGB) * T;
      const int r0 = s_r0[par][1][o], r1 = s_r1[par][1][o], stp = s_cs[par][1][o];
      const ST* ptr = static_cast<const ST*>(Bp) + s_base[par][1][o] + (long long)c0 * stp +
                      (long long)i * s_is[par][1][o] + (long long)srB * s_rs[par][1][o];
      const bool rok = srB < r1;
#pragma unroll
      for (int t = 0; t < T; ++t) {
        pb[j][t] = (rok && c0 + t < r0) ? ld_raw<ST>(ptr) : 0u;
        ptr += stp;
      }
    }
#pragma unroll
    for (int j = 0; j < UPA; ++j) {
      const int w = suA + j * USA, o = w / KGA, c0 = (w % KGA) * T;
      const int r0 = s_r0[par][0][o], r1 = s_r1[par][0][o], stp = s_cs[par][0][o];
      const ST* ptr = static_cast<const ST*>(Ap) + s_base[par][0][o] + (long long)c0 * stp +
                      (long long)i * s_is[par][0][o] + (long long)srA * s_rs[par][0][o];
      const bool rok = srA < r1;
#pragma unroll
      for (int t = 0; t < T; ++t) {
        pa[j][t] = (rok && c0 + t < r0) ? ld_raw<ST>(ptr) : 0u;
        ptr += stp;
      }
    }
  };
  // registers -> slice buffer s: one 16-byte store per K run (a whole core-matrix row)
  auto store_slice = [&](int s) {
#pragma unroll
    for (int j = 0; j < UPB; ++j) {
      const int w = suB + j * USB, o = w / KGB, cg = w % KGB;
      const uint32_t off = (uint32_t)(srB >> 3) * SBOB + (uint32_t)cg * kLBO + (uint32_t)(srB & 7) * 16u;
      *reinterpret_cast<uint4*>(bsl + (s * TB + o) * SLB + off) = pack_raw<KIND, ST, T>(pb[j]);
    }
#pragma unroll
    for (int j = 0; j < UPA; ++j) {
      const int w = suA + j * USA, o = w / KGA, cg = w % KGA;
      const uint32_t off = (uint32_t)(srA >> 3) * SBOA + (uint32_t)cg * kLBO + (uint32_t)(srA & 7) * 16u;
      *reinterpret_cast<uint4*>(asl + (s * TA + o) * SLA + off) = pack_raw<KIND, ST, T>(pa[j]);
    }
  };

  // pipelined loop: MMA1 of slice j (slice buffer sb) into T buffer tb, MMA2 of slice j from
  // T copy tb and slice buffer sb
  auto issue_mma1 = [&](int sb, int tb) {
    const uint64_t da = sdesc(su32(mop), SBOB), db = sdesc(su32(bsl + sb * TB * SLB), SBOB);
#pragma unroll
    for (int b = 0; b < TB; ++b)
#pragma unroll
      for (int kk = 0; kk < RB / O::KI; ++kk)
        mma<KIND>(st.tmem + (uint32_t)tb * 256u + (uint32_t)(b * RB), da + ((b * BIGB + kk * 2 * kLBO) >> 4),
                  db + ((b * SLB + kk * 2 * kLBO) >> 4), ID1, kk > 0);
  };
  auto issue_mma2 = [&](int sb, int tb, bool acc) {
    const uint64_t da = sdesc(su32(top + tb * TA * BIGA), SBOA), db = sdesc(su32(asl + sb * TA * SLA), SBOA);
#pragma unroll
    for (int a = 0; a < TA; ++a)
#pragma unroll
      for (int kk = 0; kk < RA / O::KI; ++kk)
        mma<KIND>(st.tmem + 128u + (uint32_t)(a * RA), da + ((a * BIGA + kk * 2 * kLBO) >> 4),
                  db + ((a * SLA + kk * 2 * kLBO) >> 4), ID2, (acc || kk > 0) ? 1u : 0u);
  };

  int iter = 0;
  load_slice(0, 0);
  for (int k = 0; k < d; ++k) {
    const int n = nmode(k);
    if (k + 1 < d) fill_info(k + 1, (k + 1) & 1);  // read after the next block barrier
    if constexpr (PIPE) {
      // prologue: slice 0 -> buffer 0, its first product into T buffer 0
      store_slice(0);
      async_fence();
      tc_before();
      if (__syncthreads_or(st.bad)) return false;
      if (tid == 0) {
        tc_after();
        issue_mma1(0, 0);
      }
      pipe_commit(st, 1, 0);
      pipe_mark(st, 1, 0);
      if (n > 1)
        load_slice(k, 1);
      else if (k + 1 < d)
        load_slice(k + 1, 0);
      for (int i = 0; i < n; ++i) {
        const int p = i & 1;
        // slice i - 2's second product frees T copy p and slice buffer (i + 1) % 3
        pipe_wait(st, 2, p);
        if (i + 1 < n) {
          store_slice((i + 1) % 3);
          async_fence();
          tc_before();
          if (__syncthreads_or(st.bad)) return false;
          // slice i + 1's first product into the other T buffer (transposed in iteration i - 1)
          if (tid == 0) {
            tc_after();
            issue_mma1((i + 1) % 3, p ^ 1);
          }
          pipe_commit(st, 1, p ^ 1);
          pipe_mark(st, 1, p ^ 1);
          if (i + 2 < n)
            load_slice(k, i + 2);
          else if (k + 1 < d)
            load_slice(k + 1, 0);
        }
        pipe_wait(st, 1, p);
        tc_after();
        epi_transpose<KIND, RA, SBOA, BIGA>(st.tmem + (uint32_t)p * 256u, top + p * TA * BIGA);
        async_fence();
        tc_before();
        if (__syncthreads_or(st.bad)) return false;
        if (tid == 0) {
          tc_after();
          issue_mma2(i % 3, p, i > 0);
        }
        pipe_commit(st, 2, p);
        pipe_mark(st, 2, p);
      }
      pipe_wait(st, 2, 0);
      pipe_wait(st, 2, 1);
      tc_after();
    } else {
    for (int i = 0; i < n; ++i, ++iter) {
      const int s = NBUF == 2 ? (iter & 1) : 0;
      if (NBUF == 1 && st.pending2) {  // the single slice buffer is still read by MMA2
        st.bad |= !mbar_wait(st.bar2, st.ph2);
        st.ph2 ^= 1u;
        st.pending2 = false;
      }
      store_slice(s);
      async_fence();
      tc_before();
      if (__syncthreads_or(st.bad)) return false;
      // ---- MMA1: T for every b (TMEM columns b*RB .. b*RB + RB - 1)
      if (tid == 0) {
        tc_after();
        const uint64_t da = sdesc(su32(mop), SBOB), db = sdesc(su32(bsl + s * TB * SLB), SBOB);
#pragma unroll
        for (int b = 0; b < TB; ++b)
#pragma unroll
          for (int kk = 0; kk < RB / O::KI; ++kk)
            mma<KIND>(st.tmem + (uint32_t)(b * RB), da + ((b * BIGB + kk * 2 * kLBO) >> 4),
                      db + ((b * SLB + kk * 2 * kLBO) >> 4), ID1, kk > 0);
        mma_commit(st.bar1);
      }
      st.pending1 = true;
      // ---- prefetch the next slice while the products run
      {
        int k2 = k, i2 = i + 1;
        if (i2 == n) { ++k2; i2 = 0; }
        if (k2 < d) load_slice(k2, i2);
      }
      st.bad |= !mbar_wait(st.bar1, st.ph1);
      st.ph1 ^= 1u;
      st.pending1 = false;
      if (st.pending2) {  // T_a is still read by the previous MMA2
        st.bad |= !mbar_wait(st.bar2, st.ph2);
        st.ph2 ^= 1u;
        st.pending2 = false;
      }
      tc_after();
      // ---- epilogue 1: T (rows (a, al), cols (b, bp)) -> T_a[(b, bp), al]
      epi_transpose<KIND, RA, SBOA, BIGA>(st.tmem, top);
      async_fence();
      tc_before();
      if (__syncthreads_or(st.bad)) return false;
      // ---- MMA2: D_a += T_a A_a,i for every a (TMEM columns 128 + a*RA ..)
      if (tid == 0) {
        tc_after();
        const uint64_t da = sdesc(su32(top), SBOA), db = sdesc(su32(asl + s * TA * SLA), SBOA);
#pragma unroll
        for (int a = 0; a < TA; ++a)
#pragma unroll
          for (int kk = 0; kk < RA / O::KI; ++kk)
            mma<KIND>(st.tmem + 128u + (uint32_t)(a * RA), da + ((a * BIGA + kk * 2 * kLBO) >> 4),
                      db + ((a * SLA + kk * 2 * kLBO) >> 4), ID2, (i > 0 || kk > 0) ? 1u : 0u);
        mma_commit(st.bar2);
      }
      st.pending2 = true;
    }
    st.bad |= !mbar_wait(st.bar2, st.ph2);
    st.ph2 ^= 1u;
    st.pending2 = false;
    tc_after();
    }
    // ---- epilogue 2: D (rows (b, bp), cols (a, ap)) -> M_b[(a, ap), bp], or the Gram entries;
    // the adjoint sweeps also store D to its slot (after core k: interface k + 1, or d - 1 - k)
    if (k + 1 < d) {
      if (slots) {
        char* const o0 = slots + (size_t)((dir * d + (dir ? d - 2 - k : k + 1)) * 2) * kSlot;
        store_partial<KIND, RA, RB>(st.tmem + 128u, o0, o0 + kSlot, dir ? nullptr : st.s_g);
      }
      epi_transpose<KIND, RB, SBOB, BIGB>(st.tmem + 128u, mop);
    } else if (!slots) {
      const int b = row / RB, bp = row % RB;
#pragma unroll
      for (int cc = 0; cc < 64; cc += 16) {
        const int c0 = h * 64 + cc;
        float v[16];
        tmem_ld16(st.tmem + ((uint32_t)(q * 32) << 16) + 128u + (uint32_t)c0, v);
        if (bp == 0 && b < nb && k + 1 == d) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = c0 + j, a = col / RA;
            if (col % RA != 0 || a >= na) continue;
            if (g.mode == 0) {
              if (g.swap)
                g.out[(long long)(b0 + b) * g.ldo + (a0 + a)] = v[j];
              else
                g.out[(long long)(a0 + a) * g.ldo + (b0 + b)] = v[j];
            } else {
              const long long S = g.gstart[grp + 1] - g.gstart[grp];
              const int la = g.perm[a0 + a], lb = g.perm[b0 + b];
              float* o = g.gout + g.gout_off[grp];
              o[la * S + lb] = v[j];
              if (sym) o[lb * S + la] = v[j];
            }
          }
        }
      }
    }
    async_fence();
    tc_before();
    if (__syncthreads_or(st.bad)) return false;
    tc_after();
  }
  return true;
}

template <int KIND, int RA, int RB, typename ST, bool PIPE = false>
__device__ __forceinline__ bool mma_tile(const GramMmaArgs& g, char* sm, MmaState& st, int grp, int a0, int na,
                                         int b0, int nb, int sym, int d, int dir = 0, char* slots = nullptr) {
  return mma_tile_sync<KIND, RA, RB, ST, PIPE>(g, sm, st, grp, a0, na, b0, nb, sym, d, dir, slots);
}

// Common prologue / epilogue of the kernels: TMEM allocation, barriers, and the release of
// the tensor memory after a bounded wait for anything still in flight.
// bars: 6 mbarriers (the plain loop's two, the pipelined loop's four)
__device__ __forceinline__ void mma_setup(MmaState& st, uint64_t* bars, uint32_t* s_tmem, char* sm, uint32_t bytes,
                                          uint32_t cols = kTmemCols) {
  const int tid = threadIdx.x, warp = tid >> 5;
  for (uint32_t e = (uint32_t)tid * 16u; e < bytes; e += kMmaThreads * 16u)
    *reinterpret_cast<uint4*>(sm + e) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0)
    for (int j = 0; j < 6; ++j) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bars[j])));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(s_tmem)), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  async_fence();
  tc_before();
  __syncthreads();
  tc_after();
  st.tmem = *s_tmem;
  st.cols = cols;
  st.bar1 = su32(&bars[0]);
  st.bar2 = su32(&bars[1]);
  st.ph1 = st.ph2 = 0;
  st.pending1 = st.pending2 = false;
  for (int j = 0; j < 2; ++j) {
    st.b1[j] = su32(&bars[2 + j]);
    st.b2[j] = su32(&bars[4 + j]);
    st.q1[j] = st.q2[j] = 0;
    st.pd1[j] = st.pd2[j] = false;
  }
  st.bad = 0;
}

__device__ __forceinline__ void mma_teardown(const GramMmaArgs& g, MmaState& st, bool failed) {
  if (failed) {
    // a product did not signal completion: one more bounded wait for whatever is still in
    // flight before the tensor memory is released, and report the timeout
    if (threadIdx.x == 0 && g.err) atomicExch(g.err, (int)T3F_ERR_TIMEOUT);
    if (st.pending1) mbar_wait(st.bar1, st.ph1);
    if (st.pending2) mbar_wait(st.bar2, st.ph2);
    for (int j = 0; j < 2; ++j) {
      if (st.pd1[j]) mbar_wait(st.b1[j], st.q1[j]);
      if (st.pd2[j]) mbar_wait(st.b2[j], st.q2[j]);
    }
  }
  tc_before();
  __syncthreads();
  tc_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(st.tmem), "r"(st.cols));
}

// CTAs per SM the shared memory of a tile shape allows (at most 2: the tensor memory holds two)
__host__ __device__ constexpr int mma_ctas_per_sm(int es, int RA, int RB) {
  return mma_layout(es, RA, RB).total + 1024u <= kSmemCap / 2u ? 2 : 1;
}

// Per-CTA state of the sweep kernels besides the dynamic operand area.
struct MmaShared {
  uint64_t bar[6];
  long long base[2][2][8];
  int r0[2][2][8], r1[2][2][8], cs[2][2][8], rs[2][2][8], is[2][2][8];
  float gv[64];
  int item[8];
  uint32_t tmem;
  int valid, wi, dir;
};

__device__ __forceinline__ void mma_bind(MmaState& st, MmaShared& sh) {
  st.s_base = &sh.base[0][0][0];
  st.s_r0 = &sh.r0[0][0][0];
  st.s_r1 = &sh.r1[0][0][0];
  st.s_cs = &sh.cs[0][0][0];
  st.s_rs = &sh.rs[0][0][0];
  st.s_is = &sh.is[0][0][0];
  st.s_g = sh.gv;
}

// Uniform batches: one tile per CTA, fixed (RA, RB). With g.scr set (adjoint sweeps) the grid
// is twice the tile count: the second half runs the reversed sweeps.
template <int KIND, int RA, int RB, typename ST>
__global__ void __launch_bounds__(kMmaThreads, mma_ctas_per_sm(OpT<KIND>::ES, RA, RB)) k_gram_mma(const __grid_constant__ GramMmaArgs g) {
  extern __shared__ __align__(128) char sm[];
  __shared__ __align__(16) MmaShared sh;
  MmaState st;
  mma_bind(st, sh);
  mma_setup(st, sh.bar, &sh.tmem, sm, g.smem_bytes);
  constexpr int TA = 128 / RA, TB = 128 / RB;
  const int ntb = (g.B.batch + TB - 1) / TB, nta = (g.A.batch + TA - 1) / TA;
  const int dir = g.scr ? (int)(blockIdx.x / (unsigned)(nta * ntb)) : 0;
  const int w = (int)(blockIdx.x % (unsigned)(nta * ntb));
  const int a0 = (w / ntb) * TA, b0 = (w % ntb) * TB;
  char* const slots = g.scr ? g.scr + (size_t)w * (size_t)g.sstride * (128u * 128u * OpT<KIND>::ES) : nullptr;
  const bool ok = mma_tile<KIND, RA, RB, ST>(g, sm, st, 0, a0, min(TA, g.A.batch - a0), b0,
                                             min(TB, g.B.batch - b0), 0, g.A.d, dir, slots);
  mma_teardown(g, st, !ok);
}

// Work-list mode: persistent CTAs drain tiles of any of the six shapes RA <= RB. With g.scr set
// (adjoint sweeps) the counter runs over twice the items: item w in both directions.
template <int KIND, typename ST>
__global__ void __launch_bounds__(kMmaThreads, 1) k_gram_mma_list(const __grid_constant__ GramMmaArgs g) {
  extern __shared__ __align__(128) char sm[];
  __shared__ __align__(16) MmaShared sh;
  MmaState st;
  mma_bind(st, sh);
  constexpr bool PIPE = KIND == 1;  // the pipelined loop fits shared memory for BF16 operands
  mma_setup(st, sh.bar, &sh.tmem, sm, g.smem_bytes, PIPE ? kTmemColsPipe : kTmemCols);
  const int tid = threadIdx.x;
  const int total = g.scr ? 2 * g.nitems : g.nitems;
  bool ok = true;
  while (ok) {
    __syncthreads();
    if (tid == 0) {
      const int w = atomicAdd(g.head, 1);
      sh.valid = w < total ? 1 : 0;
      if (w < total) {
        const int wi = w % g.nitems;
        for (int x = 0; x < 8; ++x) sh.item[x] = g.items[wi * 8 + x];
        sh.wi = wi;
        sh.dir = w >= g.nitems ? 1 : 0;
      }
    }
    __syncthreads();
    if (!sh.valid) break;
    const int grp = sh.item[0], a0 = sh.item[1], na = sh.item[2], b0 = sh.item[3], nb = sh.item[4], RA = sh.item[5],
              sym = sh.item[6], RB = sh.item[7];
    const int dir = sh.dir, d = g.gd[grp];
    char* const slots = g.scr ? g.scr + (size_t)g.soff[sh.wi] * (128u * 128u * OpT<KIND>::ES) : nullptr;
    const int key = RA * 1000 + RB;
    switch (key) {
      case 16016: ok = mma_tile<KIND, 16, 16, ST, PIPE>(g, sm, st, grp, a0, na, b0, nb, sym, d, dir, slots); break;
      case 16032: ok = mma_tile<KIND, 16, 32, ST, PIPE>(g, sm, st, grp, a0, na, b0, nb, sym, d, dir, slots); break;
      case 16064: ok = mma_tile<KIND, 16, 64, ST, PIPE>(g, sm, st, grp, a0, na, b0, nb, sym, d, dir, slots); break;
      case 32032: ok = mma_tile<KIND, 32, 32, ST, PIPE>(g, sm, st, grp, a0, na, b0, nb, sym, d, dir, slots); break;
      case 32064: ok = mma_tile<KIND, 32, 64, ST, PIPE>(g, sm, st, grp, a0, na, b0, nb, sym, d, dir, slots); break;
      default: ok = mma_tile<KIND, 64, 64, ST, PIPE>(g, sm, st, grp, a0, na, b0, nb, sym, d, dir, slots); break;
    }
  }
  mma_teardown(g, st, !ok);
}

int pad_pow2_16(int r) { return r <= 16 ? 16 : (r <= 32 ? 32 : 64); }

template <int KIND, int RA, int RB, typename ST>
t3f_status launch_mma(const GramMmaArgs& g0, cudaStream_t s) {
  GramMmaArgs g = g0;
  g.smem_bytes = mma_layout(OpT<KIND>::ES, RA, RB).total;
  g.mode = 0;
  constexpr int TA = 128 / RA, TB = 128 / RB;
  const long long grid = (long long)((g.A.batch + TA - 1) / TA) * ((g.B.batch + TB - 1) / TB) * (g.scr ? 2 : 1);
  if (grid <= 0) return T3F_OK;
  if (grid > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  auto kern = k_gram_mma<KIND, RA, RB, ST>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem_bytes) != cudaSuccess)
    return T3F_ERR_CUDA;
  kern<<<(unsigned)grid, kMmaThreads, g.smem_bytes, s>>>(g);
  return launch_status();
}

template <int KIND, typename ST>
t3f_status dispatch_r(int RA, int RB, const GramMmaArgs& g, cudaStream_t s) {
  switch (RA * 1000 + RB) {
    case 16016: return launch_mma<KIND, 16, 16, ST>(g, s);
    case 16032: return launch_mma<KIND, 16, 32, ST>(g, s);
    case 16064: return launch_mma<KIND, 16, 64, ST>(g, s);
    case 32032: return launch_mma<KIND, 32, 32, ST>(g, s);
    case 32064: return launch_mma<KIND, 32, 64, ST>(g, s);
    default: return launch_mma<KIND, 64, 64, ST>(g, s);
  }
}

uint32_t list_smem(int es) {
  uint32_t m = 0;
  const int rs[3] = {16, 32, 64};
  for (int x = 0; x < 3; ++x)
    for (int y = x; y < 3; ++y)
      m = std::max(m, (es == 2 ? mma_layout_pipe(es, rs[x], rs[y]) : mma_layout(es, rs[x], rs[y])).total);
  return m;
}

template <int KIND, typename ST>
t3f_status launch_list(const GramMmaArgs& g0, cudaStream_t s) {
  GramMmaArgs g = g0;
  g.smem_bytes = list_smem(OpT<KIND>::ES);
  g.mode = 1;
  if (g.nitems <= 0) return T3F_OK;
  auto kern = k_gram_mma_list<KIND, ST>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem_bytes) != cudaSuccess)
    return T3F_ERR_CUDA;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return T3F_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMmaThreads, g.smem_bytes) != cudaSuccess)
    return T3F_ERR_CUDA;
  const int total = g.scr ? 2 * g.nitems : g.nitems;
  const int grid = std::max(1, std::min(total, sms * std::max(per_sm, 1)));
  kern<<<grid, kMmaThreads, g.smem_bytes, s>>>(g);
  return launch_status();
}

}  // namespace

// Persistent tensor-core Gram over a work list of rank-sorted ragged objects (groups mode);
// every item is a tile of (128 / RA) x (128 / RB) pairs of one group, RA <= RB.
t3f_status launch_gram_mma_list(int math, const void* cores, int dtype, int dmax, const long long* off,
                                const int* rk, const int* nmodes, const int* items, int nitems, int* head,
                                const int* gstart, const int* gd, float* gout, const long long* gout_off,
                                const int* perm, int* err, cudaStream_t s) {
  GramMmaArgs g;
  memset(&g, 0, sizeof(g));
  g.cores = cores;
  g.off = off;
  g.rk = rk;
  g.dmax = dmax;
  g.nmodes = nmodes;
  g.gd = gd;
  g.gstart = gstart;
  g.perm = perm;
  g.gout_off = gout_off;
  g.gout = gout;
  g.items = items;
  g.nitems = nitems;
  g.head = head;
  g.err = err;
  if (math == T3F_MATH_TF32) {
    if (dtype != T3F_F32) return T3F_ERR_DTYPE;
    return launch_list<0, float>(g, s);
  }
  if (dtype == T3F_BF16) return launch_list<1, __nv_bfloat16>(g, s);
  return launch_list<1, float>(g, s);
}

// Adjoint sweeps over uniform batches (A the side of the smaller padded rank; swap = the
// caller's batches were exchanged, dG stays in the caller's [a][b] order with row stride ldg):
// both directions of every tile store their partials into scr, sstride slot orientations
// per tile.
t3f_status run_gram_mma_sweeps(const TTV& A, const TTV& B, int swap, const float* dG, int ldg, int math, char* scr,
                               long long sstride, int* err, cudaStream_t s) {
  GramMmaArgs g;
  memset(&g, 0, sizeof(g));
  g.A = A;
  g.B = B;
  g.swap = swap;
  g.gcot = dG;
  g.ldg = ldg;
  g.scr = scr;
  g.sstride = sstride;
  g.err = err;
  const int ra = pad_pow2_16(A.rmax), rb = pad_pow2_16(B.rmax);
  if (math == T3F_MATH_TF32) {
    if (A.dtype != T3F_F32) return T3F_ERR_DTYPE;
    return dispatch_r<0, float>(ra, rb, g, s);
  }
  if (A.dtype == T3F_BF16) return dispatch_r<1, __nv_bfloat16>(ra, rb, g, s);
  return dispatch_r<1, float>(ra, rb, g, s);
}

// Adjoint sweeps over the tensor-core tile list of a ragged collection: item w in both
// directions (the counter runs to 2 nitems), slots of item w from soff[w]; dout holds the
// groups' cotangents like the forward's output. heads[0] must be zero.
t3f_status launch_gram_mma_sweeps_list(int math, const void* cores, int dtype, int dmax, const long long* off,
                                       const int* rk, const int* nmodes, const int* items, int nitems, int* heads,
                                       const int* gstart, const int* gd, const long long* gout_off, const int* perm,
                                       const float* dout, char* scr, const long long* soff, int* err, cudaStream_t s) {
  GramMmaArgs g;
  memset(&g, 0, sizeof(g));
  g.cores = cores;
  g.off = off;
  g.rk = rk;
  g.dmax = dmax;
  g.nmodes = nmodes;
  g.gd = gd;
  g.gstart = gstart;
  g.perm = perm;
  g.gout_off = gout_off;
  g.gcot = dout;
  g.items = items;
  g.nitems = nitems;
  g.head = heads;
  g.err = err;
  g.scr = scr;
  g.soff = soff;
  if (math == T3F_MATH_TF32) {
    if (dtype != T3F_F32) return T3F_ERR_DTYPE;
    return launch_list<0, float>(g, s);
  }
  if (dtype == T3F_BF16) return launch_list<1, __nv_bfloat16>(g, s);
  return launch_list<1, float>(g, s);
}

bool gram_mma_supported(const TTV& A, const TTV& B, int math) {
  if (math != T3F_MATH_TF32 && math != T3F_MATH_BF16) return false;
  if (A.is_matrix || B.is_matrix) return false;
  if (A.rmax > 64 || B.rmax > 64) return false;
  if (math == T3F_MATH_TF32 && (A.dtype != T3F_F32 || B.dtype != T3F_F32)) return false;
  if (A.dtype != B.dtype) return false;
  return true;
}

t3f_status run_gram_mma(const TTV& A, const TTV& B, float* out, int math, int* err, cudaStream_t s) {
  GramMmaArgs g;
  memset(&g, 0, sizeof(g));
  const int RA = pad_pow2_16(A.rmax), RB = pad_pow2_16(B.rmax);
  // the kernels take the side of the smaller padded rank as A; the output is transposed back
  g.swap = RA > RB ? 1 : 0;
  g.A = g.swap ? B : A;
  g.B = g.swap ? A : B;
  g.ldo = B.batch;
  g.out = out;
  g.err = err;
  const int ra = std::min(RA, RB), rb = std::max(RA, RB);
  if (math == T3F_MATH_TF32) return dispatch_r<0, float>(ra, rb, g, s);
  if (A.dtype == T3F_BF16) return dispatch_r<1, __nv_bfloat16>(ra, rb, g, s);
  return dispatch_r<1, float>(ra, rb, g, s);
}

}  // namespace t3f
