// Tiled Gram sweep (paper Section 4, 'gram' / 'norm'; batches of Section 3.1).
//
// A CTA owns a tile of na x nb pairs (a, b) and carries their left partials
// M^{ab} (r^A_k x r^B_k) in shared memory through the whole sweep. Per mode slice i of core k
// the update M' = sum_i A_i^T (M B_i) is two batched products with 4 x 4 register blocks:
//   GEMM1  T[a][al][b][bp]   = sum_be M[a][al][b][be] B_b,i[be][bp]     (stacked over a)
//   GEMM2  M'[a][ap][b][bp] += sum_al A_a,i[al][ap] T[a][al][b][bp]     (stacked over b)
// Ranks are zero-padded to multiples of 4 (RA, RB). The next slice is staged into a second
// shared-memory buffer with 4-byte asynchronous copies (issued by rows shared by 4-16
// threads) while the current slice computes, and the products of a core stop at the tile's
// effective ranks on that core (boundary cores, outer rank 1, cost little). The same kernel
// serves uniform batches (tile from blockIdx) and ragged, rank-bucketed groups of objects
// (tiles taken from a work list by persistent CTAs, see gram_groups.cu).
#include "t3f_internal.cuh"

namespace t3f {

// Per-object core access: uniform batch (TTV) or a table of per-object offsets and ranks.
struct ObjTable {
  const long long* off;   // [obj][d] element offset of core k
  const int* rk;          // [obj][d + 1] ranks
  int d;
};

struct GramTileArgs {
  // uniform mode
  TTV A, B;
  int TA, TB;           // tile objects (uniform mode)
  int RA, RB;           // padded ranks (uniform mode)
  // table mode (groups)
  ObjTable tab;
  const void* gcores;   // cores of all objects
  const int* nmodes;    // [group][d] modes
  const int* items;     // work list: [item][8] = group, a0, na, b0, nb, RA, RB, sym
  int nitems;
  int* head;            // queue head (table mode)
  const int* gstart;    // [group + 1] first object of each group
  const int* gd;        // [group] d of the group
  float* gout;          // [group][S][S] Gram matrices (S = objects of the group)
  const long long* gout_off;  // [group] offset of the group's matrix
  const int* perm;            // [sorted object] local index of the object within its group
  // common
  float* out;           // uniform: [bA][bB]
  int mode;             // 0 uniform, 1 table
  int dtype;
  int maxTA, maxTB, maxRA, maxRB;
};

__device__ __forceinline__ void fma44(float (&acc)[4][4], const float4 a, const float4 b) {
  const float av[4] = {a.x, a.y, a.z, a.w};
  const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
}

template <typename T>
__device__ __forceinline__ float ldv(const void* p, long long i) {
  return ldf<T>(static_cast<const T*>(p), i);
}

constexpr int kGTMaxBlk = 2;   // output blocks per thread
constexpr int kGTMaxPF = 16;   // staging elements per thread and slice

template <typename ST>
__global__ void __launch_bounds__(512) k_gram_tile(const __grid_constant__ GramTileArgs g) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_item[8];
  // per-core object info, two core parities: [side * 16 + object] core offset and ranks
  __shared__ long long s_ob[2][32];
  __shared__ int s_or0[2][32], s_or1[2][32], s_on[2];
  // effective ranks of a core over the tile's objects (padded to 4): [parity][A left, A right,
  // B left, B right]; the products skip the 4 x 4 blocks and K steps beyond them (boundary
  // cores have rank 1 on their outer side)
  __shared__ int s_er[2][4];
  // the same ranks unpadded: K loops stop there (the operands are zero beyond them, so the
  // dropped terms are exact zeros)
  __shared__ int s_ek[2][4];
  const int tid = threadIdx.x, nth = blockDim.x;

  for (int it = 0;; ++it) {
    int grp = 0, a0, na, b0, nb, RA, RB, sym = 0, d;
    if (g.mode == 0) {
      if (it > 0) break;
      const int ntb = (g.B.batch + g.TB - 1) / g.TB;
      a0 = (blockIdx.x / ntb) * g.TA;
      b0 = (blockIdx.x % ntb) * g.TB;
      na = min(g.TA, g.A.batch - a0);
      nb = min(g.TB, g.B.batch - b0);
      RA = g.RA;
      RB = g.RB;
      d = g.A.d;
    } else {
      __syncthreads();
      if (tid == 0) {
        const int w = atomicAdd(g.head, 1);
        s_item[7] = w;
        if (w < g.nitems)
          for (int q = 0; q < 7; ++q) s_item[q] = g.items[w * 8 + q];
      }
      __syncthreads();
      if (s_item[7] >= g.nitems) break;
      grp = s_item[0];
      a0 = s_item[1];
      na = s_item[2];
      b0 = s_item[3];
      nb = s_item[4];
      RA = s_item[5];
      RB = s_item[6];
      sym = g.items[s_item[7] * 8 + 7];
      d = g.gd[grp];
    }
    const int QA = RA / 4, QB = RB / 4;
    const int nblk = na * QA * nb * QB;           // 4x4 blocks of one partial tile
    // T rows are padded to whole 128-byte lines and their 16-byte units XOR-swizzled by
    // (row / 4) mod 8, so lanes storing consecutive 4-row blocks hit different banks while
    // lanes reading one row still read a permutation of consecutive units
    const int TR = ((nb * RB + 31) / 32) * 32;

    const int szM = na * RA * nb * RB;
    // shared memory of this tile: MT [nb][RB][na][RA], TT [na][RA][TR], two staging buffers
    float* MT = sm;
    float* TT = MT + szM;
    float* As = TT + (size_t)na * RA * TR;
    // initial partials: M = 1 at (al, be) = (0, 0) of every pair
    for (int e = tid; e < szM; e += nth) {
      const int al = e % RA, a = (e / RA) % na, be = (e / (RA * na)) % RB;
      MT[e] = (al == 0 && be == 0) ? 1.0f : 0.0f;
      (void)a;
    }
    // per-object access helpers
    auto objA = [&](int t, int k, long long* base, int* r0, int* r1, int* n) {
      if (g.mode == 0) {
        *base = core_base(g.A, k, a0 + t);
        *r0 = g.A.r[k];
        *r1 = g.A.r[k + 1];
        *n = g.A.n[k];
      } else {
        const int o = a0 + t;
        *base = g.tab.off[(long long)o * g.tab.d + k];
        *r0 = g.tab.rk[(long long)o * (g.tab.d + 1) + k];
        *r1 = g.tab.rk[(long long)o * (g.tab.d + 1) + k + 1];
        *n = g.nmodes[grp * g.tab.d + k];
      }
    };
    auto objB = [&](int t, int k, long long* base, int* r0, int* r1, int* n) {
      if (g.mode == 0) {
        *base = core_base(g.B, k, b0 + t);
        *r0 = g.B.r[k];
        *r1 = g.B.r[k + 1];
        *n = g.B.n[k];
      } else {
        const int o = b0 + t;
        *base = g.tab.off[(long long)o * g.tab.d + k];
        *r0 = g.tab.rk[(long long)o * (g.tab.d + 1) + k];
        *r1 = g.tab.rk[(long long)o * (g.tab.d + 1) + k + 1];
        *n = g.nmodes[grp * g.tab.d + k];
      }
    };
    const void* Ap = g.mode == 0 ? g.A.p : g.gcores;
    const void* Bp = g.mode == 0 ? g.B.p : g.gcores;
    const int szA = na * RA * RA, szS = szA + nb * RB * RB;
    // exact quotients of the line indices (< 2^10) by R through 32-bit reciprocals
    const unsigned mA = 0xffffffffu / (unsigned)RA + 1u, mB = 0xffffffffu / (unsigned)RB + 1u;
    // core offsets and ranks of the tile's objects for core k into parity slot par; the
    // slots are filled ahead of use and published by a later block barrier
    auto fill_info = [&](int k, int par) {
      if (tid < 32) {
        const int side = tid >> 4, t = tid & 15;
        long long base = 0;
        int r0 = 0, r1 = 0, n = 1;
        if (side == 0 && t < na) objA(t, k, &base, &r0, &r1, &n);
        if (side == 1 && t < nb) objB(t, k, &base, &r0, &r1, &n);
        s_ob[par][tid] = base;
        s_or0[par][tid] = r0;
        s_or1[par][tid] = r1;
        if (tid == 0) s_on[par] = n;
        int m0 = r0, m1 = r1;  // maxima over each half-warp (one side's objects)
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          m0 = max(m0, __shfl_xor_sync(0xffffffffu, m0, o));
          m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        }
        if (t == 0) {
          s_er[par][2 * side] = max(4, (m0 + 3) & ~3);
          s_er[par][2 * side + 1] = max(4, (m1 + 3) & ~3);
          s_ek[par][2 * side] = max(1, m0);
          s_ek[par][2 * side + 1] = max(1, m1);
        }
      }
    };
    // stage slice i of core k into `buf` (zero-padded): FP32 cores are copied asynchronously
    // (cp.async, 4 bytes, zero-fill outside the ranks), BF16 cores converted on the way. The
    // padded slices are cut into rows of R elements; 2^lt consecutive threads share a row, so
    // an object's offset and ranks are read once per row. lt (2, 3 or 4) minimises rows per
    // thread x (row setup + elements per thread).
    const int nlA = na * RA, nl = nlA + nb * RB;
    int lt = 4;
    {
      int best = 0x7fffffff;
      for (int c = 2; c <= 4; ++c) {
        const int lines = (nl + (nth >> c) - 1) / (nth >> c), per = (max(RA, RB) + (1 << c) - 1) >> c;
        const int cost = lines * (4 + per);
        if (cost < best) {
          best = cost;
          lt = c;
        }
      }
    }
    auto stage = [&](int k, int i, float* buf) {
      const int par = k & 1, n = s_on[par], p0 = tid & ((1 << lt) - 1);
      for (int ln = tid >> lt; ln < nl; ln += nth >> lt) {
        const int side = ln < nlA ? 0 : 1;
        const unsigned l2 = (unsigned)(side ? ln - nlA : ln), R = side ? RB : RA;
        const unsigned t = __umulhi(l2, side ? mB : mA), w = l2 - t * R;  // object, row in it
        const int slot = side * 16 + (int)t, r0 = s_or0[par][slot], r1 = s_or1[par][slot];
        const int lim = (int)w < r0 ? r1 : 0;  // columns p < lim are inside the core
        const long long idx0 = s_ob[par][slot] + ((long long)w * n + i) * r1;
        float* dst = buf + (side ? szA : 0) + (t * R + w) * R;
        const void* src = side == 0 ? Ap : Bp;
        for (int p = p0; p < (int)R; p += 1 << lt) {
          const bool ok = p < lim;
          const long long idx = ok ? idx0 + p : 0;
          if (sizeof(ST) == 4) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + p);
            const float* gp = static_cast<const float*>(src) + idx;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gp), "r"(ok ? 4 : 0));
          } else {
            dst[p] = ok ? ldv<ST>(src, idx) : 0.0f;
          }
        }
      }
      if (sizeof(ST) == 4) asm volatile("cp.async.commit_group;\n" ::);
    };
    // this thread's output blocks: GEMM1 in row-major order, GEMM2 in column-major order
    int g1m[kGTMaxBlk], g1b[kGTMaxBlk], g1t[kGTMaxBlk];
    int g2a[kGTMaxBlk], g2t[kGTMaxBlk], g2w[kGTMaxBlk];
#pragma unroll
    for (int q = 0; q < kGTMaxBlk; ++q) {
      const int blk = tid + q * nth;
      g1m[q] = g1b[q] = g1t[q] = g2a[q] = g2t[q] = g2w[q] = -1;
      if (blk < nblk) {
        {
          const int qa = blk % QA, a = (blk / QA) % na, qb = (blk / (QA * na)) % QB, b = blk / (QA * na * QB);
          g1m[q] = (b * RB * na + a) * RA + 4 * qa;
          g1b[q] = b * RB * RB + 4 * qb;
          g1t[q] = (a * RA + 4 * qa) | qb << 16;           // first T row | qb
          g1b[q] |= (b * QB + qb) << 20 | (int)((unsigned)qa << 28);  // unit = b * QB + qb | qa
        }
        {
          const int qb = blk % QB, b = (blk / QB) % nb, qa = (blk / (QB * nb)) % QA, a = blk / (QB * nb * QA);
          g2a[q] = a * RA * RA + 4 * qa;
          g2t[q] = a * RA | qb << 16;                      // T row of al = 0 | qb
          g2a[q] |= (b * QB + qb) << 20 | (int)((unsigned)qa << 28);  // unit | qa (the ap block)
          g2w[q] = ((b * RB + 4 * qb) * na + a) * RA + 4 * qa;
        }
      }
    }
    const int mstep = na * RA;
    float* stg[2] = {As, As + szS};
    int k = 0, i = 0, cur = 0;
    fill_info(0, 0);
    if (d > 1) fill_info(1, 1);
    __syncthreads();
    stage(0, 0, stg[0]);
    float acc[kGTMaxBlk][4][4];
    while (k < d) {
      const int nk = s_on[k & 1];
      if (i == 0) {
#pragma unroll
        for (int q = 0; q < kGTMaxBlk; ++q)
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[q][x][y] = 0.0f;
      }
      // issue the next slice, then wait for the current one
      {
        int k2 = k, i2 = i + 1;
        if (i2 >= nk) {
          k2 = k + 1;
          i2 = 0;
        }
        if (k2 < d) {
          stage(k2, i2, stg[cur ^ 1]);
          if (sizeof(ST) == 4) asm volatile("cp.async.wait_group 1;\n" ::);
        } else if (sizeof(ST) == 4) {
          asm volatile("cp.async.wait_group 0;\n" ::);
        }
      }
      __syncthreads();
      const float* Asb = stg[cur];
      const float* Bsb = stg[cur] + szA;
      const int eA0 = s_er[k & 1][0], eA1 = s_er[k & 1][1], eB1 = s_er[k & 1][3];
      const int kA0 = s_ek[k & 1][0], kB0 = s_ek[k & 1][2];
      // GEMM1: T[a][al][b][bp] = sum_be MT[b][be][a][al] Bs[b][be][bp]  (al < eA0, bp < eB1,
      // be < kB0)
#pragma unroll
      for (int q = 0; q < kGTMaxBlk; ++q) {
        if (g1m[q] < 0) continue;
        if (4 * (int)((unsigned)g1b[q] >> 28) >= eA0 || 4 * (g1t[q] >> 16) >= eB1) continue;
        float t4[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) t4[x][y] = 0.0f;
        const float* mrow = MT + g1m[q];
        const float* brow = Bsb + (g1b[q] & 0xfffff);
        for (int be = 0; be < kB0; ++be)
          fma44(t4, *reinterpret_cast<const float4*>(mrow + be * mstep), *reinterpret_cast<const float4*>(brow + be * RB));
        const int unit = (g1b[q] >> 20) & 0xff;
        const int row0t = g1t[q] & 0xffff;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int r = row0t + x;
          *reinterpret_cast<float4*>(TT + r * TR + 4 * (unit ^ ((r >> 2) & 7))) =
              make_float4(t4[x][0], t4[x][1], t4[x][2], t4[x][3]);
        }
      }
      __syncthreads();
      // GEMM2: acc[a][ap][b][bp] += sum_al As[a][al][ap] T[a][al][b][bp]  (ap < eA1, bp < eB1,
      // al < kA0)
#pragma unroll
      for (int q = 0; q < kGTMaxBlk; ++q) {
        if (g2w[q] < 0) continue;
        if (4 * (int)((unsigned)g2a[q] >> 28) >= eA1 || 4 * (g2t[q] >> 16) >= eB1) continue;
        const float* arow = Asb + (g2a[q] & 0xfffff);
        const int unit = (g2a[q] >> 20) & 0xff;
        const int rbase = g2t[q] & 0xffff;
        for (int al = 0; al < kA0; ++al) {
          const int r = rbase + al;
          fma44(acc[q], *reinterpret_cast<const float4*>(arow + al * RA),
                *reinterpret_cast<const float4*>(TT + r * TR + 4 * (unit ^ ((r >> 2) & 7))));
        }
      }
      if (i + 1 == nk && k + 2 < d) fill_info(k + 2, k & 1);  // core k's slices are all staged
      __syncthreads();  // stg[cur] and TT are free again
      cur ^= 1;
      if (++i >= nk) {
        // end of core k: the accumulated blocks become the next partial (transposed layout)
#pragma unroll
        for (int q = 0; q < kGTMaxBlk; ++q) {
          if (g2w[q] < 0) continue;
#pragma unroll
          for (int y = 0; y < 4; ++y)
            *reinterpret_cast<float4*>(MT + g2w[q] + y * mstep) =
                make_float4(acc[q][0][y], acc[q][1][y], acc[q][2][y], acc[q][3][y]);
        }
        i = 0;
        ++k;
      }
    }
    __syncthreads();
    // <A_a, B_b> = M_d[0][0]
    for (int p = tid; p < na * nb; p += nth) {
      const int a = p / nb, b = p % nb;
      const float v = MT[((size_t)b * RB * na + a) * RA];
      if (g.mode == 0) {
        g.out[(long long)(a0 + a) * g.B.batch + (b0 + b)] = v;
      } else {
        const int S = g.gstart[grp + 1] - g.gstart[grp];
        const int la = g.perm[a0 + a], lb = g.perm[b0 + b];
        float* o = g.gout + g.gout_off[grp];
        o[(long long)la * S + lb] = v;
        if (sym) o[(long long)lb * S + la] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------

static int pad4(int r) { return (r + 3) & ~3; }

size_t gram_tile_smem(int TA, int TB, int RA, int RB) {
  const size_t TR = ((size_t)(TB * RB + 31) / 32) * 32;
  return sizeof(float) * ((size_t)TA * RA * TB * RB + (size_t)TA * RA * TR + 2 * ((size_t)TA * RA * RA + (size_t)TB * RB * RB));
}

// Largest tile (TA = TB) whose blocks and staging fit one CTA of `threads`.
void plan_gram_tile(int RA, int RB, int batchA, int batchB, int* TA, int* TB, int* threads) {
  // cost model: pair-slots per SM of the most loaded SM (whole waves of CTAs), with a small
  // preference for larger tiles (operand reuse)
  *TA = 1;
  *TB = 1;
  *threads = 128;
  double best = 1e300;
  int sms = 152;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) sms = v;
    }
  }
  for (int ta = 1; ta <= 16 && ta <= batchA; ++ta) {
    for (int tb = 1; tb <= 16 && tb <= batchB; ++tb) {
      const int nblk = ta * (RA / 4) * tb * (RB / 4);
      for (int th = 128; th <= 512; th *= 2) {
        if (th * kGTMaxBlk < nblk) continue;
        if (ta * RA * RA + tb * RB * RB > th * kGTMaxPF) continue;
        const size_t smem = gram_tile_smem(ta, tb, RA, RB);
        if (smem > 200 * 1024) continue;
        int cps = 65536 / (th * 128);
        const int cps_smem = (int)((228 * 1024) / (smem + 2048));
        if (cps_smem < cps) cps = cps_smem;
        if (cps < 1) continue;
        const long long tiles = (long long)((batchA + ta - 1) / ta) * ((batchB + tb - 1) / tb);
        const long long per_sm = (tiles + (long long)sms * cps - 1) / ((long long)sms * cps) * cps;
        // padded work of the most loaded SM, discounted for reuse of larger tiles
        const int rounds = (nblk + th - 1) / th;               // blocks per thread (max)
        const double balance = (double)nblk / ((double)rounds * th);
        const double work = (double)per_sm * ta * tb * (1.0 + 0.5 / ta + 0.5 / tb) / balance;
        if (work < best - 1e-9) {
          best = work;
          *TA = ta;
          *TB = tb;
          *threads = th;
        }
      }
    }
  }
}

// Persistent launch over a work list of tiles of ragged objects (one CTA per SM).
t3f_status launch_gram_tile_table(const void* cores, int dtype, int dmax, const long long* off, const int* rk,
                                  const int* nmodes, const int* items, int nitems, int* head, const int* gstart,
                                  const int* gd, float* out, const long long* gout_off, const int* perm, size_t smem,
                                  cudaStream_t s) {
  GramTileArgs g;
  memset(&g, 0, sizeof(g));
  g.mode = 1;
  g.dtype = dtype;
  g.tab.off = off;
  g.tab.rk = rk;
  g.tab.d = dmax;
  g.gcores = cores;
  g.nmodes = nmodes;
  g.items = items;
  g.nitems = nitems;
  g.head = head;
  g.gstart = gstart;
  g.gd = gd;
  g.gout = out;
  g.gout_off = gout_off;
  g.perm = perm;
  if (smem > 227 * 1024) return T3F_ERR_UNSUPPORTED;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = nitems < sms ? (nitems > 0 ? nitems : 1) : sms;
  if (dtype == T3F_F32) {
    auto kern = k_gram_tile<float>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<grid, 512, smem, s>>>(g);
  } else {
    auto kern = k_gram_tile<__nv_bfloat16>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<grid, 512, smem, s>>>(g);
  }
  return launch_status();
}

bool gram_tile_supported(const TTV& A, const TTV& B) {
  const int RA = pad4(A.rmax), RB = pad4(B.rmax);
  if (RA > 64 || RB > 64) return false;
  int ta, tb, th;
  plan_gram_tile(RA, RB, A.batch, B.batch, &ta, &tb, &th);
  return ta * RA * RA + tb * RB * RB <= th * kGTMaxPF && ta * (RA / 4) * tb * (RB / 4) <= th * kGTMaxBlk;
}

t3f_status run_gram_tile(const TTV& A, const TTV& B, float* out, cudaStream_t s) {
  GramTileArgs g;
  memset(&g, 0, sizeof(g));
  g.A = A;
  g.B = B;
  g.RA = pad4(A.rmax);
  g.RB = pad4(B.rmax);
  int threads;
  plan_gram_tile(g.RA, g.RB, A.batch, B.batch, &g.TA, &g.TB, &threads);
  g.maxTA = g.TA;
  g.maxTB = g.TB;
  g.maxRA = g.RA;
  g.maxRB = g.RB;
  g.out = out;
  g.mode = 0;
  g.dtype = A.dtype;
  const size_t smem = gram_tile_smem(g.TA, g.TB, g.RA, g.RB);
  const long long grid = (long long)((A.batch + g.TA - 1) / g.TA) * ((B.batch + g.TB - 1) / g.TB);
  if (grid > 0x7fffffff) return T3F_ERR_UNSUPPORTED;
  if (A.dtype == T3F_F32) {
    auto kern = k_gram_tile<float>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<(unsigned)grid, threads, smem, s>>>(g);
  } else {
    auto kern = k_gram_tile<__nv_bfloat16>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<(unsigned)grid, threads, smem, s>>>(g);
  }
  return launch_status();
}

}  // namespace t3f
