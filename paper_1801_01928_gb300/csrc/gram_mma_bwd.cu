// Tensor-core adjoint of the Gram sweep (cotangent of sum_ab g_ab <A_a, B_b>; paper Section 4
// 'gram', batches of Section 3.1) with TF32 or BF16 operands and FP32 accumulation.
//
// For a pair (a, b) with left partials M_k and right partials R_{k+1} around core k,
//   dA_a^k[:, i, :] = sum_b g_ab M_k B_b^k[:, i, :] R_{k+1}^T,
//   dB_b^k[:, i, :] = sum_a g_ab M_k^T A_a^k[:, i, :] R_{k+1}.
// The two are the same contraction seen from either side of a tile: with x the side whose
// gradient is formed and y the other one,
//   T[(x, xi), (y, et')]  = sum_et gM[(x, xi), (y, et)] Y_y,i[et, et']        (one product per y)
//   dX_x,i[xi, xi']       = sum_(y, et') T[(x, xi), (y, et')] R[(x, xi'), (y, et')]
// where gM holds g_xy M (transposed for x = b) and R the right partials, both as 128 x 128
// operands. The partials come from the adjoint sweeps of the tensor-core forward kernel,
// which store every interface in both orientations, already rounded to the operand type and
// laid out as K-major operands (16-byte core matrices packed along K). A work item is (tile,
// core k, side): two bulk copies bring gM_k and R_{k+1} into shared memory, then every mode
// slice i of core k runs the two products. T lives in tensor memory; TF32 feeds it to the
// second product straight from there (the A operand may sit in tensor memory), BF16 copies it
// to shared memory rounded to BF16. The second product runs over all x at once (N = 128) and
// only its diagonal blocks (x, x) are read: lane (x, xi) adds columns x*RX .. of its row to
// the gradient with atomics (other tiles and items share the objects).
#include <algorithm>
#include <string.h>
#include <vector>

#include "gram_mma.cuh"

namespace t3f {

namespace {

// Roles: warps 0-3 stage the y side's slices, warp 4 (one lane) issues the products, warps 5-8
// (one per tensor-memory lane quarter) run the epilogues (and, for BF16, copy T to shared
// memory). Slices, T and the gradient product are double-buffered, so slice i+1's first
// product runs while slice i's second product and epilogue are in flight.
constexpr int kGThreads = 288;
constexpr int kGProd = 128;           // staging threads (warps 0-3)
constexpr int kGMmaWarp = 4;
constexpr uint32_t kGTmemCols = 512;  // T[b] at columns 128 b, the gradient product Q[b] at 256 + 128 b

struct GradTcArgs {
  int mode;                   // 0: uniform batches (tile, core, side from the block index), 1: work list
  TTV A, B;                   // uniform: the kernel's two sides
  int ntb, ntiles;            // uniform: tiles along B, tile count
  float* outA;                // uniform: gradients of the kernel's A / B side, packed like A / B (nullable)
  float* outB;
  // work-list mode: ragged objects in rank-sorted positions
  const void* cores;
  const long long* off;       // [pos][dmax] element offset of core k
  const int* rk;              // [pos][dmax + 1]
  int dmax;
  const int* nmodes;          // [group][dmax]
  const int* gd;              // [group] d
  const int* items;           // the sweep kernels' tiles: [item][8] group, a0, na, b0, nb, RA, sym, RB
  const int* gitems;          // [item][4]: tile, core, side, 0
  int ngitems;
  int* head;
  float* dX;                  // gradient in the layout of the ragged cores
  // scratch of the adjoint sweeps
  const char* scr;
  const long long* soff;      // work list: slot offset of each tile (in slot orientations)
  long long sstride;          // uniform: slot orientations per tile
  int* err;
  uint32_t smem_bytes;
};

struct GradShared {
  uint64_t ld;                    // the two partial copies of an item
  uint64_t sfull[2], sempty[2];   // slice ring: staged / read by the first product
  uint64_t tdone[2], tfree[2];    // T buffers: written / consumed
  uint64_t tsfull[2], tsfree[2];  // BF16 shared-memory copies of T: written / read
  uint64_t qdone[2], qfree[2];    // gradient product buffers: written / read by the epilogue
  uint64_t fin;                   // drain after a timeout
  long long ybase[8], xbase[8];
  int yrl[8], yrr[8], xrl[8], xrr[8];
  int item[8];
  uint32_t tmem;
  int valid, k, side, w;
};

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 32 lanes x 32 consecutive columns, without waiting (tcgen05.wait::ld before use)
__device__ __forceinline__ void tmem_ld32_nw(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// one lane polls (bounded), the warp follows
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Shared-memory plan for element size es and y rank RY: gM, R, two slice buffers and (BF16)
// two shared-memory copies of T.
__host__ __device__ constexpr uint32_t grad_slot(int es) { return 128u * 128u * (uint32_t)es; }
__host__ __device__ constexpr uint32_t grad_smem(int es, int RY) {
  return 2u * grad_slot(es) + 2u * 128u * (uint32_t)RY * (uint32_t)es + (es == 2 ? 2u * grad_slot(es) : 0u);
}

// One work item: the gradient of side `side` of a tile for core k. x0 / nx: the objects whose
// gradient is formed, y0 / ny: the others. gs counts the slices this CTA ran before (buffer
// index and barrier phases continue across items), nit its items. Returns false on a timeout.
template <int KIND, int RX, int RY, typename ST>
__device__ bool grad_item(const GradTcArgs& g, char* sm, GradShared& sh, uint32_t tmem, int grp, int x0, int nx,
                          int y0, int ny, int side, int k, int d, const char* slots, float* outX, uint32_t gs,
                          uint32_t nit) {
  using O = OpT<KIND>;
  constexpr int ES = O::ES, T = 16 / ES;
  constexpr int TY = 128 / RY;
  constexpr uint32_t SLOT = grad_slot(ES);
  constexpr uint32_t SBO = (128u / T) * 128u;          // full operand: bytes per 8 rows
  constexpr uint32_t SBOY = (uint32_t)(RY / T) * 128u;  // slice operand of one y: bytes per 8 rows
  constexpr uint32_t YSZ = (uint32_t)RY * RY * ES;     // bytes of one y's slice operand
  constexpr uint32_t SLICE = 128u * RY * ES;           // one slice buffer (all y)
  constexpr int KGY = RY / T, UPY = TY * RY * KGY / kGProd, USY = kGProd / RY;
  static_assert(UPY * kGProd == TY * RY * KGY, "staging split");
  constexpr uint32_t ID1 = idesc(O::FMT, RY), ID2 = idesc(O::FMT, 128);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  char* const mx = sm;
  char* const rg = sm + SLOT;
  char* const ysl = sm + 2 * SLOT;
  char* const ts = ysl + 2 * SLICE;  // BF16 only
  const ST* const Yp = static_cast<const ST*>(g.mode == 0 ? (side ? g.A.p : g.B.p) : g.cores);
  const int n = g.mode == 0 ? g.A.n[k] : g.nmodes[grp * g.dmax + k];

  // ---- the two partials: gM_k (slot k of the left sweep) and R_{k+1} (slot k of the right
  // sweep) in the orientation whose rows are this side's objects. The previous item's
  // products have completed (its epilogues waited for the last one before the item barrier).
  if (tid == kGMmaWarp * 32) {
    expect_tx(su32(&sh.ld), 2u * SLOT);
    bulk_g2s(su32(mx), slots + (size_t)(k * 2 + side) * SLOT, SLOT, su32(&sh.ld));
    bulk_g2s(su32(rg), slots + (size_t)((d + k) * 2 + side) * SLOT, SLOT, su32(&sh.ld));
  }
  // ---- objects of both sides at core k
  if (tid < 16) {
    const int o = tid & 7, isx = tid >> 3, cnt = isx ? nx : ny, o0 = isx ? x0 : y0;
    long long base = 0;
    int rl = 0, rr = 0;
    if (o < cnt) {
      if (g.mode == 0) {
        const TTV& V = (isx ? side : !side) ? g.B : g.A;
        base = V.off[k] + (long long)(o0 + o) * V.osz[k];
        rl = V.r[k];
        rr = V.r[k + 1];
      } else {
        const int pos = o0 + o;
        base = g.off[(long long)pos * g.dmax + k];
        rl = g.rk[(long long)pos * (g.dmax + 1) + k];
        rr = g.rk[(long long)pos * (g.dmax + 1) + k + 1];
      }
    }
    if (isx) {
      sh.xbase[o] = base;
      sh.xrl[o] = rl;
      sh.xrr[o] = rr;
    } else {
      sh.ybase[o] = base;
      sh.yrl[o] = rl;
      sh.yrr[o] = rr;
    }
  }
  __syncthreads();

  bool ok = true;
  if (warp < 4) {
    // ---- staging: slice i of the y side (rows et' = right rank, K = et = left rank)
    const int sy = tid % RY, uy = tid / RY;
    uint32_t py[UPY][T];
    auto load_slice = [&](int i) {
#pragma unroll
      for (int j = 0; j < UPY; ++j) {
        const int w = uy + j * USY, o = w / KGY, c0 = (w % KGY) * T;
        const int rl = sh.yrl[o], rr = sh.yrr[o], stp = n * rr;
        const ST* ptr = Yp + sh.ybase[o] + (long long)c0 * stp + (long long)i * rr + sy;
        const bool rok = sy < rr;
#pragma unroll
        for (int t = 0; t < T; ++t) {
          py[j][t] = (rok && c0 + t < rl) ? ld_raw<ST>(ptr) : 0u;
          ptr += stp;
        }
      }
    };
    load_slice(0);
    for (int i = 0; i < n; ++i) {
      const uint32_t gg = gs + (uint32_t)i, b = gg & 1u;
      if (gg >= 2u && !warp_wait(su32(&sh.sempty[b]), ((gg >> 1) - 1u) & 1u)) {
        ok = false;
        break;
      }
      char* const buf = ysl + b * SLICE;
#pragma unroll
      for (int j = 0; j < UPY; ++j) {
        const int w = uy + j * USY, o = w / KGY, cg = w % KGY;
        const uint32_t off = (uint32_t)(sy >> 3) * SBOY + (uint32_t)cg * 128u + (uint32_t)(sy & 7) * 16u;
        *reinterpret_cast<uint4*>(buf + o * YSZ + off) = pack_raw<KIND, ST, T>(py[j]);
      }
      async_fence();
      mbar_arrive(su32(&sh.sfull[b]));
      if (i + 1 < n) load_slice(i + 1);
    }
  } else if (warp == kGMmaWarp) {
    // ---- products, issued by one lane
    if (lane == 0) {
      ok = mbar_wait(su32(&sh.ld), nit & 1u);
      for (int i = 0; ok && i <= n; ++i) {
        if (i < n) {
          const uint32_t gg = gs + (uint32_t)i, b = gg & 1u;
          ok = mbar_wait(su32(&sh.sfull[b]), (gg >> 1) & 1u);
          if (ok && gg >= 2u) ok = mbar_wait(su32(&sh.tfree[b]), ((gg >> 1) - 1u) & 1u);
          if (!ok) break;
          tc_after();
          // T[(x, xi), (y, et')] = sum_et gM[(x, xi), (y, et)] Y_y,i[et, et'] for every y
#pragma unroll
          for (int y = 0; y < TY; ++y)
#pragma unroll
            for (int kk = 0; kk < RY / O::KI; ++kk) {
              const uint64_t da = sdesc2(su32(mx) + (uint32_t)((y * RY + kk * O::KI) / T) * 128u, 128u, SBO);
              const uint64_t db = sdesc2(su32(ysl + b * SLICE) + (uint32_t)y * YSZ + (uint32_t)(kk * O::KI / T) * 128u,
                                         128u, SBOY);
              mma<KIND>(tmem + b * 128u + (uint32_t)(y * RY), da, db, ID1, kk > 0 ? 1u : 0u);
            }
          mma_commit(su32(&sh.tdone[b]));
          mma_commit(su32(&sh.sempty[b]));
        }
        if (i >= 1) {
          // T R^T over all x at once (N = 128, K = 128) into Q[bj]; only its diagonal blocks
          // (x, x) are read -- the same products as one N = RX product per x, in 128 / KI
          // instructions instead of TX times as many
          const uint32_t gj = gs + (uint32_t)(i - 1), bj = gj & 1u;
          ok = mbar_wait(su32(KIND == 0 ? &sh.tdone[bj] : &sh.tsfull[bj]), (gj >> 1) & 1u);
          if (ok && gj >= 2u) ok = mbar_wait(su32(&sh.qfree[bj]), ((gj >> 1) - 1u) & 1u);
          if (!ok) break;
          tc_after();
#pragma unroll
          for (int kk = 0; kk < 128 / O::KI; ++kk) {
            const uint64_t db = sdesc2(su32(rg) + (uint32_t)(kk * O::KI / T) * 128u, 128u, SBO);
            if constexpr (KIND == 0) {
              mma_ts_tf32(tmem + 256u + bj * 128u, tmem + bj * 128u + (uint32_t)(kk * O::KI), db, ID2, kk > 0 ? 1u : 0u);
            } else {
              const uint64_t da = sdesc2(su32(ts + bj * SLOT) + (uint32_t)(kk * O::KI / T) * 128u, 128u, SBO);
              mma<KIND>(tmem + 256u + bj * 128u, da, db, ID2, kk > 0 ? 1u : 0u);
            }
          }
          mma_commit(su32(&sh.qdone[bj]));
          mma_commit(su32(KIND == 0 ? &sh.tfree[bj] : &sh.tsfree[bj]));
        }
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue warps: lane quarter qd of tensor memory
    const int qd = warp & 3, row = qd * 32 + lane, xr = row / RX, xi = row % RX;
    constexpr int QCOLS = RX < 32 ? 32 : RX;  // columns of the x blocks this quarter's lanes cover
    const int cstart = ((qd * 32) / RX) * RX;
    const bool xok = xr < nx && xi < sh.xrl[xr];
    const int xrr = sh.xrr[xr];
    const long long xrow = sh.xbase[xr] + (long long)xi * n * xrr;
    for (int i = 0; i <= n; ++i) {
      if constexpr (KIND == 1) {
        if (i < n) {
          // T(i) -> shared memory (rows (x, xi), K = (y, et')), rounded to BF16
          const uint32_t gg = gs + (uint32_t)i, b = gg & 1u;
          if (!warp_wait(su32(&sh.tdone[b]), (gg >> 1) & 1u) ||
              (gg >= 2u && !warp_wait(su32(&sh.tsfree[b]), ((gg >> 1) - 1u) & 1u))) {
            ok = false;
            break;
          }
          tc_after();
          char* const dst = ts + b * SLOT;
#pragma unroll
          for (int cc = 0; cc < 128; cc += 64) {
            uint32_t r[2][32];
            tmem_ld32_nw(tmem + b * 128u + ((uint32_t)(qd * 32) << 16) + (uint32_t)cc, r[0]);
            tmem_ld32_nw(tmem + b * 128u + ((uint32_t)(qd * 32) << 16) + (uint32_t)(cc + 32), r[1]);
            tmem_wait_ld();
#pragma unroll
            for (int hh = 0; hh < 8; ++hh) {
              float u[8];
#pragma unroll
              for (int t = 0; t < 8; ++t) u[t] = __uint_as_float(r[hh >> 2][(hh & 3) * 8 + t]);
              *reinterpret_cast<uint4*>(dst + (uint32_t)(row >> 3) * SBO + (uint32_t)((cc + hh * 8) / 8) * 128u +
                                        (uint32_t)(row & 7) * 16u) = O::pack(u);
            }
          }
          async_fence();
          tc_before();
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(su32(&sh.tsfull[b]));
            mbar_arrive(su32(&sh.tfree[b]));
          }
        }
      }
      const int j = KIND == 0 ? i : i - 1;  // slice whose epilogue runs now
      if (j < 0 || j >= n) continue;
      const uint32_t gj = gs + (uint32_t)j, bj = gj & 1u;
      if (!warp_wait(su32(&sh.qdone[bj]), (gj >> 1) & 1u)) {
        ok = false;
        break;
      }
      tc_after();
      // lane (x, xi) adds its block's columns to dX_x[xi, j, :]
      uint32_t r[QCOLS / 32][32];
#pragma unroll
      for (int h = 0; h < QCOLS / 32; ++h)
        tmem_ld32_nw(tmem + 256u + bj * 128u + ((uint32_t)(qd * 32) << 16) + (uint32_t)(cstart + h * 32), r[h]);
      tmem_wait_ld();
      if (xok && outX) {
        float* const dst = outX + xrow + (long long)j * xrr;
#pragma unroll
        for (int t = 0; t < QCOLS; ++t) {
          const int c = cstart + t, xc = c / RX, xp = c % RX;
          if (xc == xr && xp < xrr) atomicAdd(dst + xp, __uint_as_float(r[t >> 5][t & 31]));
        }
      }
      tc_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(su32(&sh.qfree[bj]));
    }
  }
  return ok;
}

template <int KIND>
__device__ __forceinline__ void grad_setup(GradShared& sh, char* sm, uint32_t bytes) {
  const int tid = threadIdx.x, warp = tid >> 5;
  for (uint32_t e = (uint32_t)tid * 16u; e < bytes; e += kGThreads * 16u)
    *reinterpret_cast<uint4*>(sm + e) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    auto init = [](uint64_t* b, uint32_t count) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
    };
    init(&sh.ld, 1);
    init(&sh.fin, 1);
    for (int b = 0; b < 2; ++b) {
      init(&sh.sfull[b], kGProd);
      init(&sh.sempty[b], 1);
      init(&sh.tdone[b], 1);
      init(&sh.tfree[b], KIND == 0 ? 1 : 4);
      init(&sh.tsfull[b], 4);
      init(&sh.tsfree[b], 1);
      init(&sh.qdone[b], 1);
      init(&sh.qfree[b], 4);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sh.tmem)),
                 "r"(kGTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  async_fence();
  tc_before();
  __syncthreads();
  tc_after();
}

__device__ __forceinline__ void grad_teardown(const GradTcArgs& g, GradShared& sh, bool failed, uint32_t nit) {
  if (failed) {
    // a wait ran out: report it, then let whatever is still in flight finish (bounded) before
    // the tensor memory is released -- the products through one more commit, the last copy
    if (threadIdx.x == 0 && g.err) atomicExch(g.err, (int)T3F_ERR_TIMEOUT);
    if (threadIdx.x == kGMmaWarp * 32) {
      mma_commit(su32(&sh.fin));
      mbar_wait(su32(&sh.fin), 0);
      if (nit > 0) mbar_wait(su32(&sh.ld), (nit - 1u) & 1u);
    }
  }
  tc_before();
  __syncthreads();
  tc_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh.tmem), "r"(kGTmemCols));
}

template <int KIND, typename ST>
__device__ bool grad_dispatch(const GradTcArgs& g, char* sm, GradShared& sh, int grp, int a0, int na, int b0, int nb,
                              int RA, int RB, int side, int k, int d, const char* slots, float* outX, uint32_t gs,
                              uint32_t nit) {
  const int x0 = side ? b0 : a0, nx = side ? nb : na, y0 = side ? a0 : b0, ny = side ? na : nb;
  const int RX = side ? RB : RA, RY = side ? RA : RB;
  const uint32_t tm = sh.tmem;
#define T3F_GRAD_CASE(rx, ry)                                                                                  \
  case rx * 1000 + ry:                                                                                         \
    return grad_item<KIND, rx, ry, ST>(g, sm, sh, tm, grp, x0, nx, y0, ny, side, k, d, slots, outX, gs, nit);
  switch (RX * 1000 + RY) {
    T3F_GRAD_CASE(16, 16)
    T3F_GRAD_CASE(16, 32)
    T3F_GRAD_CASE(16, 64)
    T3F_GRAD_CASE(32, 16)
    T3F_GRAD_CASE(32, 32)
    T3F_GRAD_CASE(32, 64)
    T3F_GRAD_CASE(64, 16)
    T3F_GRAD_CASE(64, 32)
    default:
      return grad_item<KIND, 64, 64, ST>(g, sm, sh, tm, grp, x0, nx, y0, ny, side, k, d, slots, outX, gs, nit);
  }
#undef T3F_GRAD_CASE
}

// Uniform batches: block = (tile, core, side); work list: persistent CTAs drain (tile, core,
// side) items through an atomic counter.
template <int KIND, typename ST>
__global__ void __launch_bounds__(kGThreads, 1) k_gram_tc_grad(const __grid_constant__ GradTcArgs g) {
  extern __shared__ __align__(128) char sm[];
  __shared__ __align__(16) GradShared sh;
  grad_setup<KIND>(sh, sm, g.smem_bytes);
  constexpr uint32_t SLOT = grad_slot(OpT<KIND>::ES);
  const int tid = threadIdx.x;
  bool failed = false;
  uint32_t gs = 0, nit = 0;
  if (g.mode == 0) {
    const int d = g.A.d;
    const int w = blockIdx.x / (2 * d), k = (blockIdx.x / 2) % d, side = blockIdx.x % 2;
    float* const outX = side ? g.outB : g.outA;
    if (outX) {
      const int RA = g.A.rmax <= 16 ? 16 : (g.A.rmax <= 32 ? 32 : 64);
      const int RB = g.B.rmax <= 16 ? 16 : (g.B.rmax <= 32 ? 32 : 64);
      const int TA = 128 / RA, TB = 128 / RB;
      const int a0 = (w / g.ntb) * TA, b0 = (w % g.ntb) * TB;
      const char* slots = g.scr + (size_t)w * (size_t)g.sstride * SLOT;
      const bool ok = grad_dispatch<KIND, ST>(g, sm, sh, 0, a0, min(TA, g.A.batch - a0), b0, min(TB, g.B.batch - b0),
                                              RA, RB, side, k, d, slots, outX, gs, nit);
      nit = 1;
      failed = __syncthreads_or(!ok) != 0;
    }
  } else {
    while (true) {
      __syncthreads();
      if (tid == 0) {
        const int w = atomicAdd(g.head, 1);
        sh.valid = w < g.ngitems ? 1 : 0;
        if (w < g.ngitems) {
          const int t = g.gitems[w * 4];
          sh.w = t;
          sh.k = g.gitems[w * 4 + 1];
          sh.side = g.gitems[w * 4 + 2];
          for (int x = 0; x < 8; ++x) sh.item[x] = g.items[t * 8 + x];
        }
      }
      __syncthreads();
      if (!sh.valid) break;
      const int grp = sh.item[0], a0 = sh.item[1], na = sh.item[2], b0 = sh.item[3], nb = sh.item[4], RA = sh.item[5],
                RB = sh.item[7];
      const int k = sh.k, side = sh.side, d = g.gd[grp];
      const char* slots = g.scr + (size_t)g.soff[sh.w] * SLOT;
      const bool ok = grad_dispatch<KIND, ST>(g, sm, sh, grp, a0, na, b0, nb, RA, RB, side, k, d, slots, g.dX, gs, nit);
      gs += (uint32_t)g.nmodes[grp * g.dmax + k];
      ++nit;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
  }
  grad_teardown(g, sh, failed, nit);
}

uint32_t grad_smem_max(int es) { return grad_smem(es, 64); }

template <int KIND, typename ST>
t3f_status launch_grad(const GradTcArgs& g0, int grid, cudaStream_t s) {
  GradTcArgs g = g0;
  g.smem_bytes = grad_smem_max(OpT<KIND>::ES);
  if (grid <= 0) return T3F_OK;
  auto kern = k_gram_tc_grad<KIND, ST>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem_bytes) != cudaSuccess)
    return T3F_ERR_CUDA;
  kern<<<grid, kGThreads, g.smem_bytes, s>>>(g);
  return launch_status();
}

template <typename F>
t3f_status by_math(int math, int dtype, F&& f) {
  if (math == T3F_MATH_TF32) {
    if (dtype != T3F_F32) return T3F_ERR_DTYPE;
    return f(std::integral_constant<int, 0>{}, (float*)nullptr);
  }
  if (dtype == T3F_BF16) return f(std::integral_constant<int, 1>{}, (__nv_bfloat16*)nullptr);
  return f(std::integral_constant<int, 1>{}, (float*)nullptr);
}

}  // namespace

// sweeps of gram_mma.cu
t3f_status run_gram_mma_sweeps(const TTV& A, const TTV& B, int swap, const float* dG, int ldg, int math, char* scr,
                               long long sstride, int* err, cudaStream_t s);
t3f_status launch_gram_mma_sweeps_list(int math, const void* cores, int dtype, int dmax, const long long* off,
                                       const int* rk, const int* nmodes, const int* items, int nitems, int* head,
                                       const int* gstart, const int* gd, const long long* gout_off, const int* perm,
                                       const float* dout, char* scr, const long long* soff, int* err, cudaStream_t s);

// Slot orientations (128 x 128 operands) one tile of a uniform pair of batches keeps: both
// directions, d interfaces each, two orientations.
long long gram_tc_bwd_slots(const TTV& A) { return 4LL * A.d; }

size_t gram_tc_bwd_tiles(const TTV& A, const TTV& B) {
  const int RA = A.rmax <= 16 ? 16 : (A.rmax <= 32 ? 32 : 64), RB = B.rmax <= 16 ? 16 : (B.rmax <= 32 ? 32 : 64);
  const bool swap = RA > RB;
  const int ra = std::min(RA, RB), rb = std::max(RA, RB);
  const TTV& KA = swap ? B : A;
  const TTV& KB = swap ? A : B;
  return (size_t)((KA.batch + 128 / ra - 1) / (128 / ra)) * (size_t)((KB.batch + 128 / rb - 1) / (128 / rb));
}

// Workspace of the uniform tensor-core adjoint: the error word, then the slots (TF32 size,
// which also covers BF16).
size_t ws_gram_bwd_tc(const TTV& A, const TTV& B) {
  return kWsHeader + gram_tc_bwd_tiles(A, B) * (size_t)gram_tc_bwd_slots(A) * 128u * 128u * 4u;
}

// Uniform tensor-core adjoint: the sweeps into the scratch, then the gradient products.
// dA / dB (nullable) are zeroed here. scr must hold gram_tc_bwd_tiles * gram_tc_bwd_slots
// orientations of 128 x 128 x 4 bytes.
t3f_status run_gram_tc_backward(const TTV& A, const TTV& B, const float* dG, float* dA, float* dB, int math,
                                char* scr, int* err, cudaStream_t s) {
  const int RA = A.rmax <= 16 ? 16 : (A.rmax <= 32 ? 32 : 64), RB = B.rmax <= 16 ? 16 : (B.rmax <= 32 ? 32 : 64);
  const int swap = RA > RB ? 1 : 0;
  const TTV& KA = swap ? B : A;
  const TTV& KB = swap ? A : B;
  if (dA && cudaMemsetAsync(dA, 0, sizeof(float) * (size_t)(A.off[A.d - 1] + (long long)A.batch * A.osz[A.d - 1]), s) != cudaSuccess)
    return T3F_ERR_CUDA;
  if (dB && cudaMemsetAsync(dB, 0, sizeof(float) * (size_t)(B.off[B.d - 1] + (long long)B.batch * B.osz[B.d - 1]), s) != cudaSuccess)
    return T3F_ERR_CUDA;
  if (A.batch == 0 || B.batch == 0) return T3F_OK;
  const long long sstride = gram_tc_bwd_slots(A);
  T3F_CHECK(run_gram_mma_sweeps(KA, KB, swap, dG, B.batch, math, scr, sstride, err, s));
  GradTcArgs g;
  memset(&g, 0, sizeof(g));
  g.mode = 0;
  g.A = KA;
  g.B = KB;
  const int TB = 128 / std::max(RA, RB);
  g.ntb = (KB.batch + TB - 1) / TB;
  g.ntiles = (int)gram_tc_bwd_tiles(A, B);
  g.outA = swap ? dB : dA;
  g.outB = swap ? dA : dB;
  g.scr = scr;
  g.sstride = sstride;
  g.err = err;
  const long long grid = (long long)g.ntiles * A.d * 2;
  if (grid > 0x7fffffffLL) return T3F_ERR_UNSUPPORTED;
  return by_math(math, A.dtype, [&](auto kind, auto* st) -> t3f_status {
    using ST = std::remove_pointer_t<decltype(st)>;
    return launch_grad<decltype(kind)::value, ST>(g, (int)grid, s);
  });
}

// Work-list tensor-core adjoint over a ragged collection: the sweeps over the tensor-core tile
// list (both directions), then the (tile, core, side) gradient items. dX must be zeroed.
t3f_status launch_gram_tc_backward_list(int math, const void* cores, int dtype, int dmax, const long long* off,
                                        const int* rk, const int* nmodes, const int* items, int nitems,
                                        const int* gitems, int ngitems, int* heads, const int* gstart,
                                        const int* gd, const long long* gout_off, const int* perm,
                                        const float* dout, float* dX, char* scr, const long long* soff, int* err,
                                        cudaStream_t s) {
  if (nitems <= 0) return T3F_OK;
  T3F_CHECK(launch_gram_mma_sweeps_list(math, cores, dtype, dmax, off, rk, nmodes, items, nitems, heads, gstart, gd,
                                        gout_off, perm, dout, scr, soff, err, s));
  GradTcArgs g;
  memset(&g, 0, sizeof(g));
  g.mode = 1;
  g.cores = cores;
  g.off = off;
  g.rk = rk;
  g.dmax = dmax;
  g.nmodes = nmodes;
  g.gd = gd;
  g.items = items;
  g.gitems = gitems;
  g.ngitems = ngitems;
  g.head = heads + 1;
  g.dX = dX;
  g.scr = scr;
  g.soff = soff;
  g.err = err;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return T3F_ERR_CUDA;
  const int grid = std::max(1, std::min(ngitems, sms));
  return by_math(math, dtype, [&](auto kind, auto* st) -> t3f_status {
    using ST = std::remove_pointer_t<decltype(st)>;
    return launch_grad<decltype(kind)::value, ST>(g, grid, s);
  });
}

}  // namespace t3f
