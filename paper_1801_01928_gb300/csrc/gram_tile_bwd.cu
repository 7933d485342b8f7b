// Tiled adjoint of the Gram sweep (cotangent of sum_ab g_ab <A_a, B_b>).
//
// For a pair (a, b) with left partials M_k and right partials R_{k+1} (interfaces k, k+1):
//   dA_a^k[:, i, :] += g_ab M_k B_b^k[:, i, :] R_{k+1}^T,   dB_b^k[:, i, :] += g_ab M_k^T A_a^k[:, i, :] R_{k+1},
//   R_k = sum_i A_a^k[:, i, :] R_{k+1} B_b^k[:, i, :]^T.
// A CTA owns a tile of na x nb pairs. It first runs the left sweep of its pairs (as the
// forward kernel) and keeps M at every interface in a per-CTA scratch area, then runs the
// right sweep; per mode slice five register-blocked products (4 x 4 blocks) run on shared
// memory:
//   X  = A_i R          Y' = g B_i R^T        R' += X B_i^T
//   dA_a,i = sum_b M Y'   (K = the tile's (b, beta))      dB_b,i = sum_a (g M)^T X   (K = (a, alpha))
// dA / dB of a slice are added to the global gradients with atomics (other tiles share the
// objects). Ranks are zero-padded to multiples of 4; the same kernel takes tiles from the
// block index (uniform batches) or from a work list (grouped ragged collections).
//
// Every tile has at most one 4 x 4 block of a partial tile per thread. Block indices come
// from per-tile decode tables in shared memory; the products of a core stop at the tile's
// effective ranks on that core (the largest rank of its objects, padded to 4), so the
// boundary cores (outer rank 1) cost little. Where a phase has fewer blocks than threads,
// K ranges are split across threads of different warps (left sweep: T and M' halves; right
// sweep: R' and dA / dB parts chosen per tile by a K-step count). Core slices are staged by
// lines (rows, or columns when transposed) shared by 4-16 threads with 4-byte asynchronous
// copies, into two buffers, or into one for tiles that fit half an SM only that way (the next
// slice is then issued after a slice's last barrier). The kernel runs with 512 threads (one
// CTA per SM) or 256 (two per SM, tiles of half an SM's shared memory).
#include "t3f_internal.cuh"

namespace t3f {

struct GramBwdTileArgs {
  TTV A, B;              // uniform mode
  int TA, TB, RA, RB;
  const float* dG;       // uniform: [bA][bB]
  float* dA;             // uniform: packed like A
  float* dB;             // uniform: packed like B
  // table mode
  const long long* off;
  const int* rk;
  int dmax;
  const void* gcores;
  const int* nmodes;
  const int* items;      // [item][8]: group, a0, na, b0, nb, RA, RB, sym
  int nitems;
  int* head;
  const int* gd;
  const int* perm;
  const float* dout;     // [group][S][S]
  const long long* gout_off;
  const int* gstart;
  float* dX;             // gradient with the layout of the ragged cores
  // common
  float* scratch;        // per CTA: (dmax + 1) interfaces of the tile's partials
  long long scratch_stride;
  int mode, dtype;
};

__device__ __forceinline__ void fma44b(float (&acc)[4][4], const float4 a, const float4 b) {
  const float av[4] = {a.x, a.y, a.z, a.w};
  const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
}

constexpr int kGTBMaxPF = 16;  // staging elements per thread and slice (tiles up to 8192 elements)

// Every tile has at most as many 4 x 4 blocks of a partial tile as the CTA has threads, so a
// thread holds the accumulators of one block (a second would cost registers and spills).
constexpr int MAXB = 1;

template <typename ST>
__global__ void __launch_bounds__(512) k_gram_tile_bwd(const __grid_constant__ GramBwdTileArgs g) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_item[8];
  // per-core object info, two core parities: [side * 16 + object] core offset and ranks
  __shared__ long long s_ob[2][32];
  __shared__ int s_or0[2][32], s_or1[2][32], s_on[2];
  // effective ranks of a core over the tile's objects (padded to 4): [parity][A left, A right,
  // B left, B right]; products skip the 4 x 4 blocks and K steps beyond them (boundary cores
  // have rank 1 on their outer side)
  __shared__ int s_er[2][4];
  // the same ranks unpadded: K loops stop there (the operands are zero beyond them, so the
  // dropped terms are exact zeros)
  __shared__ int s_ek[2][4];
  const int tid = threadIdx.x, nth = blockDim.x;
  float* scr = g.scratch + (long long)blockIdx.x * g.scratch_stride;
  for (int it = 0;; ++it) {
    int grp = 0, a0, na, b0, nb, RA, RB, sym = 0, single = 0, d;
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
      const int fl = g.items[s_item[7] * 8 + 7];  // bit 0: symmetrise, bit 1: one staging buffer
      sym = fl & 1;
      single = (fl >> 1) & 1;
      d = g.gd[grp];
    }
    const int P = na * nb, PS = RA * RB, QA = RA / 4, QB = RB / 4;
    // shared memory of this tile
    float* Rm = sm;                      // [p][RA][RB]  R (rows alpha')
    float* RT = Rm + P * PS;             // [p][RB][RA]  R^T
    float* Mm = RT + P * PS;             // [a][al][b][be] g * M   (K rows (a, al) for dB)
    float* MT = Mm + P * PS;             // [b][be][a][al] M       (K rows (b, be) for dA)
    float* Xm = MT + P * PS;             // [a][al][b][bp] X       (K rows (a, al) for dB)
    float* XT = Xm + P * PS;             // [p][bp][al]    X^T     (K rows bp for R'; the 4-float
                                         // column chunk c of row bp sits at chunk (c + bp/4) mod RA/4)
    float* Ym = XT + P * PS;             // [b][be][a][ap] g Y     (K rows (b, be) for dA)
    float* Sg = Ym + P * PS;             // staging: [2 or 1][AT (na RA RA) + BT (nb RB RB)]
    const int szA = na * RA * RA, szS = szA + nb * RB * RB;
    // with one staging buffer (tiles that fit half an SM only that way) the next slice is
    // issued after the slice's last barrier and waited for at the next slice's start
    float* gsm = Sg + (single ? 1 : 2) * szS;  // [P] cotangents of the tile's pairs
    // block decode tables (a | qa << 4 | b << 8 | qb << 12), filled once per tile so that the
    // per-slice phases need no integer division: dP = pair-layout 4 x 4 blocks (qb fastest,
    // then b, qa, a), dY = Y-layout blocks (qa fastest, then a, qb, b), d3 = gradient blocks
    // (dA: a | qa << 4 | qp << 8, qp fastest; then dB: b | qb << 4 | qp << 8)
    const int nblk = na * QA * nb * QB, nda = na * QA * QA, ndb = nb * QB * QB;
    int* dP = reinterpret_cast<int*>(gsm + P);
    int* dY = dP + nblk;
    int* d3 = dY + nblk;
    int* sp = d3 + nda + ndb;  // [nth] this thread's R' / dA-dB assignment of the right sweep
    // per-object access
    auto objX = [&](int side, int t, int k, long long* base, int* r0, int* r1, int* n) {
      if (g.mode == 0) {
        const TTV& V = side == 0 ? g.A : g.B;
        *base = core_base(V, k, (side == 0 ? a0 : b0) + t);
        *r0 = V.r[k];
        *r1 = V.r[k + 1];
        *n = V.n[k];
      } else {
        const int o = (side == 0 ? a0 : b0) + t;
        *base = g.off[(long long)o * g.dmax + k];
        *r0 = g.rk[(long long)o * (g.dmax + 1) + k];
        *r1 = g.rk[(long long)o * (g.dmax + 1) + k + 1];
        *n = g.nmodes[grp * g.dmax + k];
      }
    };
    const void* Ap = g.mode == 0 ? g.A.p : g.gcores;
    const void* Bp = g.mode == 0 ? g.B.p : g.gcores;
    // cotangents of the pairs (table mode: symmetrised for off-diagonal tiles)
    for (int p = tid; p < P; p += nth) {
      const int a = p / nb, b = p % nb;
      float v;
      if (g.mode == 0) {
        v = g.dG[(long long)(a0 + a) * g.B.batch + (b0 + b)];
      } else {
        const int S = g.gstart[grp + 1] - g.gstart[grp];
        const int la = g.perm[a0 + a], lb = g.perm[b0 + b];
        const float* o = g.dout + g.gout_off[grp];
        v = o[(long long)la * S + lb];
        if (sym) v += o[(long long)lb * S + la];
      }
      gsm[p] = v;
    }
    for (int j = tid; j < nblk; j += nth) {
      {
        const int qb = j % QB, b = (j / QB) % nb, qa = (j / (QB * nb)) % QA, a = j / (QB * nb * QA);
        dP[j] = a | qa << 4 | b << 8 | qb << 12;
      }
      {
        const int qa = j % QA, a = (j / QA) % na, qb = (j / (QA * na)) % QB, b = j / (QA * na * QB);
        dY[j] = a | qa << 4 | b << 8 | qb << 12;
      }
    }
    for (int j = tid; j < nda + ndb; j += nth) {
      if (j < nda) {
        d3[j] = j / (QA * QA) | ((j / QA) % QA) << 4 | (j % QA) << 8;
      } else {
        const int bl = j - nda;
        d3[j] = bl / (QB * QB) | ((bl / QB) % QB) << 4 | (bl % QB) << 8;
      }
    }
    // core offsets and ranks of the tile's objects for core k into parity slot par; the
    // slots are filled ahead of use and published by the barrier that ends a core
    auto fill_info = [&](int k, int par) {
      if (tid < 32) {
        const int side = tid >> 4, t = tid & 15;
        long long base = 0;
        int r0 = 0, r1 = 0, n = 1;
        if (t < (side ? nb : na)) objX(side, t, k, &base, &r0, &r1, &n);
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
    // exact quotients of the line indices (< 2^10) by R through 32-bit reciprocals
    const unsigned mA = 0xffffffffu / (unsigned)RA + 1u, mB = 0xffffffffu / (unsigned)RB + 1u;
    // stage slice i of core k: trans = 0 -> [t][row][col], trans = 1 -> [t][col][row]. The
    // padded slices are cut into lines of R elements (rows, or columns when transposed);
    // 2^lt consecutive threads share a line, so an object's offset and ranks are read once
    // per line. lt (2, 3 or 4) minimises lines per thread x (line setup + elements per thread).
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
    auto stage = [&](int k, int i, float* buf, int trans) {
      const int par = k & 1, n = s_on[par], p0 = tid & ((1 << lt) - 1);
      for (int ln = tid >> lt; ln < nl; ln += nth >> lt) {
        const int side = ln < nlA ? 0 : 1;
        const unsigned l2 = (unsigned)(side ? ln - nlA : ln), R = side ? RB : RA;
        const unsigned t = __umulhi(l2, side ? mB : mA), w = l2 - t * R;  // object, line in it
        const int slot = side * 16 + (int)t, r0 = s_or0[par][slot], r1 = s_or1[par][slot];
        // element p of the line: row p (transposed) or column p; valid below lim
        const bool lok = (int)w < (trans ? r1 : r0);
        const int lim = lok ? (trans ? r0 : r1) : 0;
        const long long stride = trans ? (long long)n * r1 : 1;
        const long long idx0 = s_ob[par][slot] + (trans ? (long long)i * r1 + w : ((long long)w * n + i) * r1);
        float* dst = buf + (side ? szA : 0) + (t * R + w) * R;
        const void* src = side == 0 ? Ap : Bp;
        for (int p = p0; p < (int)R; p += 1 << lt) {
          const bool ok = p < lim;
          const long long idx = ok ? idx0 + p * stride : 0;
          if (sizeof(ST) == 4) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + p);
            const float* gp = static_cast<const float*>(src) + idx;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gp), "r"(ok ? 4 : 0));
          } else {
            dst[p] = ok ? ldf<ST>(static_cast<const ST*>(src), idx) : 0.0f;
          }
        }
      }
      if (sizeof(ST) == 4) asm volatile("cp.async.commit_group;\n" ::);
    };
    auto nmode = [&](int k) { return s_on[k & 1]; };
    fill_info(0, 0);
    if (d > 1) fill_info(1, 1);
    __syncthreads();
    // ---------------- left sweep: M at every interface into the CTA scratch ------------
    // scratch layout per interface j: [a][al][b][be]
    for (int e = tid; e < P * PS; e += nth) {
      const int be = e % RB, b = (e / RB) % nb, al = (e / (RB * nb)) % RA, a = e / (RB * nb * RA);
      const float v = (al == 0 && be == 0) ? 1.0f : 0.0f;
      scr[e] = v;  // M_0 of every pair
      MT[(((size_t)b * RB + be) * na + a) * RA + al] = v;  // MT holds M^T during the left sweep
    }
    {
      int k = 0, i = 0, cur = 0;
      stage(0, 0, Sg, 0);
      float acc[MAXB][4][4];
      // with at most half as many 4 x 4 blocks as threads, two threads share a block and split
      // its K range (T: be, M': al); their partial sums of M' are combined at the end of a core
      const int ks = 2 * nblk <= nth ? 2 : 1;
      const int hb = tid / nblk, bb = tid % nblk;  // split mode: half and block of this thread
      float* T1 = Xm;                                // second half of T in split mode
      while (k < d) {
        const int nk = nmode(k);
        if (i == 0) {
#pragma unroll
          for (int q = 0; q < MAXB; ++q)
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
              for (int y = 0; y < 4; ++y) acc[q][x][y] = 0.0f;
        }
        int k2 = k, i2 = i + 1;
        if (i2 >= nk) {
          k2 = k + 1;
          i2 = 0;
        }
        if (k2 < d && !single) {
          stage(k2, i2, Sg + (cur ^ 1) * szS, 0);
          if (sizeof(ST) == 4) asm volatile("cp.async.wait_group 1;\n" ::);
        } else if (sizeof(ST) == 4) {
          asm volatile("cp.async.wait_group 0;\n" ::);
        }
        __syncthreads();
        const float* As = Sg + cur * szS;  // [a][al][ap]
        const float* Bs = As + szA;        // [b][be][bp]
        const int eA0 = s_er[k & 1][0], eA1 = s_er[k & 1][1], eB1 = s_er[k & 1][3];
        const int kA0 = s_ek[k & 1][0], kB0 = s_ek[k & 1][2];
        // T[a][al][b][bp] = sum_be M[a][al][b][be] B[b][be][bp]  (T in RT's storage; in split
        // mode the second half of the be range goes to T1); al < eA0, bp < eB1, be < kB0
        for (int blk = ks == 2 ? bb : tid; blk < nblk && hb < ks; blk += (ks == 2 ? nblk : nth)) {
          const int dv = dP[blk], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
          if (4 * qa >= eA0 || 4 * qb >= eB1) {
            if (ks == 2) break;
            continue;
          }
          const int be0 = ks == 2 ? hb * (kB0 / 2) : 0, be1 = (ks == 2 && hb == 0) ? kB0 / 2 : kB0;
          float t4[4][4];
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) t4[x][y] = 0.0f;
          const float* mt = MT + ((size_t)b * RB * na + a) * RA + 4 * qa;  // + be * na * RA
          for (int be = be0; be < be1; ++be)
            fma44b(t4, *reinterpret_cast<const float4*>(mt + (size_t)be * na * RA),
                   *reinterpret_cast<const float4*>(Bs + ((size_t)b * RB + be) * RB + 4 * qb));
          float* tdst = (ks == 2 && hb == 1) ? T1 : RT;
#pragma unroll
          for (int x = 0; x < 4; ++x)
            *reinterpret_cast<float4*>(tdst + (((size_t)a * RA + 4 * qa + x) * nb + b) * RB + 4 * qb) =
                make_float4(t4[x][0], t4[x][1], t4[x][2], t4[x][3]);
          if (ks == 2) break;
        }
        __syncthreads();
        // M'[a][ap][b][bp] += sum_al A[a][al][ap] T[a][al][b][bp]; ap < eA1, bp < eB1, al < kA0
        if (ks == 2) {
          const int dv = dP[bb], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
          if (hb < 2 && 4 * qa < eA1 && 4 * qb < eB1) {
            const int al0 = hb * (kA0 / 2), al1 = hb == 0 ? kA0 / 2 : kA0;
            for (int al = al0; al < al1; ++al) {
              const size_t o = (((size_t)a * RA + al) * nb + b) * RB + 4 * qb;
              const float4 t0 = *reinterpret_cast<const float4*>(RT + o);
              const float4 t1 = *reinterpret_cast<const float4*>(T1 + o);
              fma44b(acc[0], *reinterpret_cast<const float4*>(As + ((size_t)a * RA + al) * RA + 4 * qa),
                     make_float4(t0.x + t1.x, t0.y + t1.y, t0.z + t1.z, t0.w + t1.w));
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < MAXB; ++q) {
            const int blk = tid + q * nth;
            if (blk < nblk) {
              const int dv = dP[blk], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
              const int al1 = (4 * qa < eA1 && 4 * qb < eB1) ? kA0 : 0;
              for (int al = 0; al < al1; ++al)
                fma44b(acc[q], *reinterpret_cast<const float4*>(As + ((size_t)a * RA + al) * RA + 4 * qa),
                       *reinterpret_cast<const float4*>(RT + (((size_t)a * RA + al) * nb + b) * RB + 4 * qb));
            }
          }
        }
        __syncthreads();
        if (single) {
          if (k2 < d) stage(k2, i2, Sg, 0);  // every thread is past its last read of the buffer
        } else {
          cur ^= 1;
        }
        if (++i >= nk) {
          // split mode: the second halves hand their partial sums to the first halves
          if (ks == 2) {
            if (hb == 1) {
              const int dv = dP[bb], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
#pragma unroll
              for (int x = 0; x < 4; ++x)
                *reinterpret_cast<float4*>(Ym + (((size_t)a * RA + 4 * qa + x) * nb + b) * RB + 4 * qb) =
                    make_float4(acc[0][x][0], acc[0][x][1], acc[0][x][2], acc[0][x][3]);
            }
            __syncthreads();
            if (hb == 0) {
              const int dv = dP[bb], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
#pragma unroll
              for (int x = 0; x < 4; ++x) {
                const float4 v = *reinterpret_cast<const float4*>(Ym + (((size_t)a * RA + 4 * qa + x) * nb + b) * RB + 4 * qb);
                acc[0][x][0] += v.x;
                acc[0][x][1] += v.y;
                acc[0][x][2] += v.z;
                acc[0][x][3] += v.w;
              }
            }
          }
#pragma unroll
          for (int q = 0; q < MAXB; ++q) {
            const int blk = ks == 2 ? (q == 0 && hb == 0 ? bb : nblk) : tid + q * nth;
            if (blk < nblk) {
              const int dv = dP[blk], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
#pragma unroll
              for (int x = 0; x < 4; ++x) {
                const size_t o = (((size_t)a * RA + 4 * qa + x) * nb + b) * RB + 4 * qb;
                *reinterpret_cast<float4*>(scr + (size_t)(k + 1) * P * PS + o) =
                    make_float4(acc[q][x][0], acc[q][x][1], acc[q][x][2], acc[q][x][3]);
              }
#pragma unroll
              for (int y = 0; y < 4; ++y)  // M^T for the next core
                *reinterpret_cast<float4*>(MT + (((size_t)b * RB + 4 * qb + y) * na + a) * RA + 4 * qa) =
                    make_float4(acc[q][0][y], acc[q][1][y], acc[q][2][y], acc[q][3][y]);
            }
          }
          if (k + 2 < d) fill_info(k + 2, k & 1);  // core k's slices are all staged
          __syncthreads();
          i = 0;
          ++k;
        }
      }
    }
    __syncthreads();
    // ---------------- right sweep with the gradient products ---------------------------
    // Per slice, R' (nblk blocks, K = RB) and dA / dB (nda + ndb blocks, K = nb RB / na RA)
    // share one barrier interval. Small tiles leave most threads idle there, so the K range
    // of a block may be split among s2 (R') or s3 (dA / dB) threads of different warps: part
    // p of block j runs on thread p * (block count rounded up to a warp) + j, so the lanes of a
    // warp still read the same K row. R' parts keep their sums in registers until the end of
    // the core; each dA / dB part adds its own sum to the gradient. The dA / dB items are
    // counted from warp off3 on, past the warps that hold R' blocks. s2, s3 minimise the
    // largest per-thread number of K steps; a split is taken only when it fits one round.
    int l2 = 0, l3 = 0;
    {
      const int nrw = (nblk + 31) & ~31, n3b = nda + ndb, n3w = (n3b + 31) & ~31;
      const int K3 = max(nb * RB, na * RA);
      int best = 0x7fffffff, off3 = 0;
      for (int a2 = 0; a2 <= 2; ++a2) {
        const int c2 = 1 << a2;
        if (c2 > 1 && (c2 * nrw > nth || QB % c2 != 0)) break;
        const int u2 = c2 == 1 ? min(nblk, nth) : c2 * nrw;
        const int load2 = c2 == 1 ? ((nblk + nth - 1) / nth) * RB : RB / c2;
        const int o3 = (u2 & ~31) % nth, f = nth - o3;
        for (int a3 = 0; a3 <= 2; ++a3) {
          const int c3 = 1 << a3;
          if (c3 > 1 && (c3 * n3w > nth || K3 < 8 * c3)) break;
          const int n3 = c3 == 1 ? n3b : c3 * n3w, k3 = K3 / c3 + (c3 > 1 ? 2 : 0);
          const int cb = (n3 + nth - 1) / nth, ca = n3 > f ? (n3 - f + nth - 1) / nth : 0;
          int m = max(cb * k3, load2 + ca * k3);
          if (u2 > o3) m = max(m, load2 + cb * k3);
          if (m < best) {
            best = m;
            l2 = a2;
            l3 = a3;
            off3 = o3;
          }
        }
      }
      // sp[tid]: low half = R' part << 12 | block (0xffff: none; unused without a split),
      // high half = dA / dB part << 12 | block, or without a split the first item index
      int v2 = 0xffff, v3;
      const int tr = (tid + nth - off3) % nth;
      if (l2 > 0) {
        const int part = tid / nrw, blk = tid - part * nrw;
        if (part < (1 << l2) && blk < nblk) v2 = part << 12 | blk;
      }
      if (l3 > 0) {
        const int part = tr / n3w, blk = tr - part * n3w;
        v3 = (part < (1 << l3) && blk < n3b) ? (part << 12 | blk) : 0xffff;
      } else {
        v3 = tr;
      }
      sp[tid] = (int)((unsigned)v2 | (unsigned)v3 << 16);  // read back by this thread only
    }
    const int s2 = 1 << l2, s3 = 1 << l3;
    // R at interface d = 1
    for (int e = tid; e < P * PS; e += nth) {
      const int q = e % PS;
      Rm[e] = q == 0 ? 1.0f : 0.0f;
      RT[e] = q == 0 ? 1.0f : 0.0f;
    }
    for (int k = d - 1; k >= 0; --k) {
      const int nk = nmode(k);
      // M at interface k, one 4 x 4 block per step: Mm = g M in [a][al][b][be], MT = M in
      // [b][be][a][al]
      for (int j = tid; j < nblk; j += nth) {
        const int dv = dP[j], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
        const float gg = gsm[a * nb + b];
        float4 v[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const size_t o = (((size_t)a * RA + 4 * qa + x) * nb + b) * RB + 4 * qb;
          v[x] = *reinterpret_cast<const float4*>(scr + (size_t)k * P * PS + o);
          *reinterpret_cast<float4*>(Mm + o) = make_float4(gg * v[x].x, gg * v[x].y, gg * v[x].z, gg * v[x].w);
        }
        float* mt = MT + (((size_t)b * RB + 4 * qb) * na + a) * RA + 4 * qa;
        *reinterpret_cast<float4*>(mt) = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
        *reinterpret_cast<float4*>(mt + (size_t)na * RA) = make_float4(v[0].y, v[1].y, v[2].y, v[3].y);
        *reinterpret_cast<float4*>(mt + (size_t)2 * na * RA) = make_float4(v[0].z, v[1].z, v[2].z, v[3].z);
        *reinterpret_cast<float4*>(mt + (size_t)3 * na * RA) = make_float4(v[0].w, v[1].w, v[2].w, v[3].w);
      }
      float racc[MAXB][4][4];
      const int nr = na * QA * nb * QB;
#pragma unroll
      for (int q = 0; q < MAXB; ++q)
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) racc[q][x][y] = 0.0f;
      int cur = 0;
      stage(k, 0, Sg, 1);
      for (int i = 0; i < nk; ++i) {
        if (i + 1 < nk && !single) {
          stage(k, i + 1, Sg + (cur ^ 1) * szS, 1);
          if (sizeof(ST) == 4) asm volatile("cp.async.wait_group 1;\n" ::);
        } else if (sizeof(ST) == 4) {
          asm volatile("cp.async.wait_group 0;\n" ::);
        }
        __syncthreads();
        const float* AT = Sg + cur * szS;  // [a][ap][al]  (A_i transposed)
        const float* BT = AT + szA;        // [b][bp][be]  (B_i transposed)
        const int eA0 = s_er[k & 1][0], eA1 = s_er[k & 1][1], eB0 = s_er[k & 1][2], eB1 = s_er[k & 1][3];
        const int kA1 = s_ek[k & 1][1], kB1 = s_ek[k & 1][3];
        // (1) X[a][al][b][bp] = sum_ap A[al][ap] R[ap][bp] (al < eA0, bp < eB1, ap < kA1);
        //     Y'[b][be][a][ap] = g sum_bp B[be][bp] R[ap][bp] (be < eB0, ap < eA1, bp < kB1)
        const int nx = na * QA * nb * QB, ny = nb * QB * na * QA;
        for (int blk = tid; blk < nx + ny; blk += nth) {
          float t4[4][4];
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) t4[x][y] = 0.0f;
          if (blk < nx) {
            const int dv = dP[blk], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
            if (4 * qa >= eA0 || 4 * qb >= eB1) continue;
            const float* rr = Rm + (size_t)(a * nb + b) * PS + 4 * qb;  // + ap * RB
            const float* at = AT + (size_t)a * RA * RA + 4 * qa;        // + ap * RA
            for (int ap = 0; ap < kA1; ++ap)
              fma44b(t4, *reinterpret_cast<const float4*>(at + ap * RA), *reinterpret_cast<const float4*>(rr + ap * RB));
#pragma unroll
            for (int x = 0; x < 4; ++x)
              *reinterpret_cast<float4*>(Xm + (((size_t)a * RA + 4 * qa + x) * nb + b) * RB + 4 * qb) =
                  make_float4(t4[x][0], t4[x][1], t4[x][2], t4[x][3]);
            // X^T rows 4qb..4qb+3: chunk qa rotated by qb spreads a warp's stores over the banks
            int cx = qa + qb;
            while (cx >= QA) cx -= QA;
#pragma unroll
            for (int y = 0; y < 4; ++y)
              *reinterpret_cast<float4*>(XT + ((size_t)(a * nb + b) * RB + 4 * qb + y) * RA + 4 * cx) =
                  make_float4(t4[0][y], t4[1][y], t4[2][y], t4[3][y]);
          } else {
            const int bl = blk - nx;
            const int dv = dY[bl], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
            if (4 * qb >= eB0 || 4 * qa >= eA1) continue;
            const float* rt = RT + (size_t)(a * nb + b) * PS + 4 * qa;  // + bp * RA
            const float* bt = BT + (size_t)b * RB * RB + 4 * qb;        // + bp * RB
            for (int bp = 0; bp < kB1; ++bp)
              fma44b(t4, *reinterpret_cast<const float4*>(bt + bp * RB), *reinterpret_cast<const float4*>(rt + bp * RA));
            const float gg = gsm[a * nb + b];
#pragma unroll
            for (int x = 0; x < 4; ++x)
              *reinterpret_cast<float4*>(Ym + (((size_t)b * RB + 4 * qb + x) * na + a) * RA + 4 * qa) =
                  make_float4(gg * t4[x][0], gg * t4[x][1], gg * t4[x][2], gg * t4[x][3]);
          }
        }
        __syncthreads();
        // (2) R'[a][al][b][be] += sum_bp X[al][bp] B[be][bp]  (bp range split s2 ways)
#pragma unroll
        for (int q = 0; q < MAXB; ++q) {
          int blk, part = 0;
          if (s2 == 1) {
            blk = tid + q * nth;
          } else {
            const int v2 = sp[tid] & 0xffff;
            blk = (q == 0 && v2 != 0xffff) ? (v2 & 0xfff) : nr;
            part = v2 >> 12;
          }
          if (blk < nr) {
            const int dv = dP[blk], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
            if (4 * qa >= eA0 || 4 * qb >= eB0) continue;  // al < eA0, be < eB0, bp < eB1
            const float* xt = XT + (size_t)(a * nb + b) * PS;     // + bp * RA + rotated chunk
            const float* bt = BT + (size_t)b * RB * RB + 4 * qb;  // + bp * RB
            const int nbq = eB1 >> 2, bq0 = (part * nbq) >> l2, bq1 = ((part + 1) * nbq) >> l2;
            int cx = qa + bq0;  // chunk of X^T column block qa in rows 4bq..4bq+3
            while (cx >= QA) cx -= QA;
            for (int bq = bq0; bq < bq1; ++bq) {
#pragma unroll
              for (int y = 0; y < 4; ++y) {
                const int bp = 4 * bq + y;
                fma44b(racc[q], *reinterpret_cast<const float4*>(xt + bp * RA + 4 * cx),
                       *reinterpret_cast<const float4*>(bt + bp * RB));
              }
              if (++cx == QA) cx = 0;
            }
          }
        }
        // (3) dA_a,i[al][ap] = sum_{b,be} M[al][be] Y'[be][ap];  dB_b,i[be][bp] = sum_{a,al} gM[al][be] X[al][bp]
        const int v3 = (int)((unsigned)sp[tid] >> 16);
        for (int w = s3 == 1 ? v3 : 0; s3 == 1 ? w < nda + ndb : (w == 0 && v3 != 0xffff); w += (s3 == 1 ? nth : 1)) {
          const int blk = s3 == 1 ? w : (v3 & 0xfff), part = s3 == 1 ? 0 : v3 >> 12;
          float t4[4][4];
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) t4[x][y] = 0.0f;
          if (blk < nda) {
            const int dv = d3[blk], qp = dv >> 8, qa = (dv >> 4) & 15, a = dv & 15;
            if (4 * qa >= eA0 || 4 * qp >= eA1) continue;  // al < eA0, ap < eA1, be < eB0
            if (eB0 == RB) {
              const int KK = nb * RB, kk1 = ((part + 1) * KK) >> l3;
              for (int kk = (part * KK) >> l3; kk < kk1; ++kk)
                fma44b(t4, *reinterpret_cast<const float4*>(MT + ((size_t)kk * na + a) * RA + 4 * qa),
                       *reinterpret_cast<const float4*>(Ym + ((size_t)kk * na + a) * RA + 4 * qp));
            } else if (part == 0) {
              for (int b = 0; b < nb; ++b)
                for (int be = 0; be < eB0; ++be) {
                  const size_t kk = (size_t)b * RB + be;
                  fma44b(t4, *reinterpret_cast<const float4*>(MT + (kk * na + a) * RA + 4 * qa),
                         *reinterpret_cast<const float4*>(Ym + (kk * na + a) * RA + 4 * qp));
                }
            }
            // core k's object info (slot k & 1, filled before the core's first slice)
            const long long base = s_ob[k & 1][a];
            const int r0 = s_or0[k & 1][a], r1 = s_or1[k & 1][a], n = nk;
            float* dst = g.mode == 0 ? g.dA : g.dX;
            if (dst)
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
              for (int y = 0; y < 4; ++y) {
                const int al = 4 * qa + x, ap = 4 * qp + y;
                if (al < r0 && ap < r1 && t4[x][y] != 0.0f) atomicAdd(dst + base + ((long long)al * n + i) * r1 + ap, t4[x][y]);
              }
          } else {
            const int dv = d3[blk], qp = dv >> 8, qb = (dv >> 4) & 15, b = dv & 15;
            if (4 * qb >= eB0 || 4 * qp >= eB1) continue;  // be < eB0, bp < eB1, al < eA0
            if (eA0 == RA) {
              const int KK = na * RA, kk1 = ((part + 1) * KK) >> l3;
              for (int kk = (part * KK) >> l3; kk < kk1; ++kk)
                fma44b(t4, *reinterpret_cast<const float4*>(Mm + ((size_t)kk * nb + b) * RB + 4 * qb),
                       *reinterpret_cast<const float4*>(Xm + ((size_t)kk * nb + b) * RB + 4 * qp));
            } else if (part == 0) {
              for (int a = 0; a < na; ++a)
                for (int al = 0; al < eA0; ++al) {
                  const size_t kk = (size_t)a * RA + al;
                  fma44b(t4, *reinterpret_cast<const float4*>(Mm + (kk * nb + b) * RB + 4 * qb),
                         *reinterpret_cast<const float4*>(Xm + (kk * nb + b) * RB + 4 * qp));
                }
            }
            const long long base = s_ob[k & 1][16 + b];
            const int r0 = s_or0[k & 1][16 + b], r1 = s_or1[k & 1][16 + b], n = nk;
            float* dst = g.mode == 0 ? g.dB : g.dX;
            if (dst)
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
              for (int y = 0; y < 4; ++y) {
                const int be = 4 * qb + x, bp = 4 * qp + y;
                if (be < r0 && bp < r1 && t4[x][y] != 0.0f) atomicAdd(dst + base + ((long long)be * n + i) * r1 + bp, t4[x][y]);
              }
          }
        }
        __syncthreads();
        if (single) {
          if (i + 1 < nk) stage(k, i + 1, Sg, 1);  // every thread is past its last read of the buffer
        } else {
          cur ^= 1;
        }
      }
      // R at interface k; with an R' split, parts 1.. hand their sums to part 0 through the
      // free X / X^T / Y buffers (nblk blocks of 16 values each, at most three parts)
      int rblk = nr;
      if (s2 > 1) {
        const int v2 = sp[tid] & 0xffff, part = v2 >> 12, blk = v2 & 0xfff;
        if (v2 != 0xffff && part > 0) {
          float* xb = part == 1 ? Xm : (part == 2 ? XT : Ym);
#pragma unroll
          for (int x = 0; x < 4; ++x)
            *reinterpret_cast<float4*>(xb + ((size_t)blk * 4 + x) * 4) =
                make_float4(racc[0][x][0], racc[0][x][1], racc[0][x][2], racc[0][x][3]);
        }
        __syncthreads();
        if (v2 != 0xffff && part == 0) {
          rblk = blk;
          for (int pp = 1; pp < s2; ++pp) {
            const float* xb = pp == 1 ? Xm : (pp == 2 ? XT : Ym);
#pragma unroll
            for (int x = 0; x < 4; ++x) {
              const float4 v = *reinterpret_cast<const float4*>(xb + ((size_t)blk * 4 + x) * 4);
              racc[0][x][0] += v.x;
              racc[0][x][1] += v.y;
              racc[0][x][2] += v.z;
              racc[0][x][3] += v.w;
            }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < MAXB; ++q) {
        const int blk = s2 == 1 ? tid + q * nth : (q == 0 ? rblk : nr);
        if (blk < nr) {
          const int dv = dP[blk], qb = dv >> 12, b = (dv >> 8) & 15, qa = (dv >> 4) & 15, a = dv & 15;
#pragma unroll
          for (int x = 0; x < 4; ++x)
            *reinterpret_cast<float4*>(Rm + (size_t)(a * nb + b) * PS + (4 * qa + x) * RB + 4 * qb) =
                make_float4(racc[q][x][0], racc[q][x][1], racc[q][x][2], racc[q][x][3]);
#pragma unroll
          for (int y = 0; y < 4; ++y)
            *reinterpret_cast<float4*>(RT + (size_t)(a * nb + b) * PS + (4 * qb + y) * RA + 4 * qa) =
                make_float4(racc[q][0][y], racc[q][1][y], racc[q][2][y], racc[q][3][y]);
        }
      }
      if (k > 0) fill_info(k - 1, (k - 1) & 1);  // core k's slices are all staged
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------------------

static int pad4b(int r) { return (r + 3) & ~3; }

size_t gram_tile_bwd_smem(int na, int nb, int RA, int RB, bool single) {
  const size_t P = (size_t)na * nb, PS = (size_t)RA * RB;
  const size_t szS = (size_t)na * RA * RA + (size_t)nb * RB * RB;
  const size_t QA = RA / 4, QB = RB / 4;
  const size_t tables = 2 * P * QA * QB + na * QA * QA + nb * QB * QB + 512;  // decode + split tables
  return sizeof(float) * (7 * P * PS + (single ? 1 : 2) * szS + P) + sizeof(int) * tables;
}

constexpr size_t kGTBMaxSmem = 220 * 1024;

bool gram_tile_bwd_fits(int na, int nb, int RA, int RB) {
  return na * RA * RA + nb * RB * RB <= 512 * kGTBMaxPF && gram_tile_bwd_smem(na, nb, RA, RB, false) <= kGTBMaxSmem;
}

// A tile for the half-size CTAs (256 threads, two CTAs per SM): at most one 4 x 4 block per
// thread and half of an SM's shared memory.
constexpr size_t kGTBSmallSmem = 110 * 1024;

bool gram_tile_bwd_fits_small(int na, int nb, int RA, int RB, bool single) {
  return na * (RA / 4) * nb * (RB / 4) <= 256 && gram_tile_bwd_smem(na, nb, RA, RB, single) <= kGTBSmallSmem;
}

// Relative throughput of the half-size form (two 256-thread CTAs per SM, whose barrier and
// load waits overlap) against one 512-thread CTA per SM on the same work.
constexpr double kGTBHalfGain = 1.15;

// Tile of a uniform batch: the balanced tile with the least work per SM, as full-size CTAs
// (512 threads, one per SM) or half-size ones (256 threads, two per SM, half an SM's shared
// memory with two staging buffers); one 4 x 4 block per thread either way.
void plan_gram_tile_bwd(int RA, int RB, int batchA, int batchB, int* TA, int* TB, int* threads) {
  *TA = 1;
  *TB = 1;
  *threads = 512;
  double best = 1e300;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int half = 0; half <= 1; ++half)
    for (int ta = 1; ta <= 16 && ta <= batchA; ++ta)
      for (int tb = 1; tb <= 16 && tb <= batchB; ++tb) {
        if (half ? !gram_tile_bwd_fits_small(ta, tb, RA, RB, false)
                 : (ta * (RA / 4) * tb * (RB / 4) > 512 || !gram_tile_bwd_fits(ta, tb, RA, RB)))
          continue;
        const long long tiles = (long long)((batchA + ta - 1) / ta) * ((batchB + tb - 1) / tb);
        const long long slots = half ? 2LL * sms : sms;
        const long long rounds = (tiles + slots - 1) / slots;
        // per-SM work: rounds x tile work (staging shared by the tile's pairs), two CTAs' worth
        // per round for the half-size form at its higher throughput
        double work = (double)rounds * ta * tb * (1.0 + 0.5 / ta + 0.5 / tb);
        if (half) work *= 2.0 / kGTBHalfGain;
        if (work < best - 1e-9) {
          best = work;
          *TA = ta;
          *TB = tb;
          *threads = half ? 256 : 512;
        }
      }
}

bool gram_tile_bwd_supported(const TTV& A, const TTV& B) {
  const int RA = pad4b(A.rmax), RB = pad4b(B.rmax);
  return RA <= 64 && RB <= 64 && gram_tile_bwd_fits(1, 1, RA, RB) &&
         A.d <= T3F_MAX_D;
}

size_t ws_gram_tile_bwd(const TTV& A, const TTV& B) {
  const int RA = pad4b(A.rmax), RB = pad4b(B.rmax);
  int ta, tb, th;
  plan_gram_tile_bwd(RA, RB, A.batch, B.batch, &ta, &tb, &th);
  const long long tiles = (long long)((A.batch + ta - 1) / ta) * ((B.batch + tb - 1) / tb);
  const long long stride = (long long)(A.d + 1) * ta * tb * RA * RB;
  return kWsHeader + align256(sizeof(float) * stride * tiles);
}

t3f_status run_gram_tile_bwd(const TTV& A, const TTV& B, const float* dG, float* dA, float* dB, void* ws,
                             size_t ws_bytes, cudaStream_t s) {
  T3F_CHECK(check_ws(ws, ws_bytes, ws_gram_tile_bwd(A, B)));
  GramBwdTileArgs g;
  memset(&g, 0, sizeof(g));
  g.A = A;
  g.B = B;
  g.RA = pad4b(A.rmax);
  g.RB = pad4b(B.rmax);
  int threads;
  plan_gram_tile_bwd(g.RA, g.RB, A.batch, B.batch, &g.TA, &g.TB, &threads);
  g.dG = dG;
  g.dA = dA;
  g.dB = dB;
  g.mode = 0;
  g.dtype = A.dtype;
  g.scratch = reinterpret_cast<float*>(static_cast<char*>(ws) + kWsHeader);
  g.scratch_stride = (long long)(A.d + 1) * g.TA * g.TB * g.RA * g.RB;
  const size_t smem = gram_tile_bwd_smem(g.TA, g.TB, g.RA, g.RB, false);
  const long long grid = (long long)((A.batch + g.TA - 1) / g.TA) * ((B.batch + g.TB - 1) / g.TB);
  auto go = [&](auto kern) -> t3f_status {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<(unsigned)grid, threads, smem, s>>>(g);
    return T3F_OK;
  };
  T3F_CHECK(A.dtype == T3F_F32 ? go(k_gram_tile_bwd<float>) : go(k_gram_tile_bwd<__nv_bfloat16>));
  return launch_status();
}

// Persistent adjoint over a work list of ragged tiles (grouped Gram matrices).
t3f_status launch_gram_tile_bwd_table(const void* cores, int dtype, int dmax, const long long* off, const int* rk,
                                      const int* nmodes, const int* items, int nitems, int* head, const int* gstart,
                                      const int* gd, const int* perm, const float* dout, const long long* gout_off,
                                      float* dX, float* scratch, long long scratch_stride, size_t smem, int grid,
                                      int threads, cudaStream_t s) {
  GramBwdTileArgs g;
  memset(&g, 0, sizeof(g));
  g.mode = 1;
  g.dtype = dtype;
  g.off = off;
  g.rk = rk;
  g.dmax = dmax;
  g.gcores = cores;
  g.nmodes = nmodes;
  g.items = items;
  g.nitems = nitems;
  g.head = head;
  g.gstart = gstart;
  g.gd = gd;
  g.perm = perm;
  g.dout = dout;
  g.gout_off = gout_off;
  g.dX = dX;
  g.scratch = scratch;
  g.scratch_stride = scratch_stride;
  if (smem > 227 * 1024) return T3F_ERR_UNSUPPORTED;
  // the list's tiles have at most one 4 x 4 block per thread
  auto go = [&](auto kern) -> t3f_status {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return T3F_ERR_CUDA;
    kern<<<grid, threads, smem, s>>>(g);
    return T3F_OK;
  };
  T3F_CHECK(dtype == T3F_F32 ? go(k_gram_tile_bwd<float>) : go(k_gram_tile_bwd<__nv_bfloat16>));
  return launch_status();
}

}  // namespace t3f
