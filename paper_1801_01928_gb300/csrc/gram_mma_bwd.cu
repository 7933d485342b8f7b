// Tensor-core adjoint of the Gram sweep (cotangent of sum_ab g_ab <A_a, B_b>; paper Section 4
// 'gram', batches of Section 3.1) with TF32 or BF16 operands and FP32 accumulation.
//
// For a pair (a, b) with left partials M_k and right partials R_{k+1} around core k,
//   dA_a^k[:, i, :] = sum_b g_ab M_k B_b^k[:, i, :] R_{k+1}^T,
//   dB_b^k[:, i, :] = sum_a g_ab M_k^T A_a^k[:, i, :] R_{k+1}.
// The two are the same contraction seen from either side of a tile: with x the side whose
// gradient is formed and y the other one,
//   T[(x, xi), (y, et')]  = sum_et gM[(x, xi), (y, et)] Y_y,i[et, et']        (one product per y)
//   dX_x,i[xi, xi']       = sum_(y, et') T[(x, xi), (y, et')] R[(x, xi'), (y, et')]   (one per x)
// where gM holds g_xy M (transposed for x = b) and R the right partials, both as 128 x 128
// operands. The partials come from the adjoint sweeps of the tensor-core forward kernel,
// which store every interface in both orientations, already rounded to the operand type and
// laid out as K-major operands (16-byte core matrices packed along K). A work item is (tile,
// core k, side): two bulk copies bring gM_k and R_{k+1} into shared memory, then every mode
// slice i of core k runs the two products. T lives in tensor memory; TF32 feeds it to the
// second product straight from there (the A operand may sit in tensor memory), BF16 copies it
// to shared memory rounded to BF16. Only the lanes of block x of the second product's output
// belong to object x; they are added to the gradient with atomics (other tiles and items
// share the objects).
#include <algorithm>
#include <string.h>
#include <vector>

#include "gram_mma.cuh"

namespace t3f {

namespace {

constexpr int kGThreads = 256;
constexpr uint32_t kGTmemCols = 256;  // T at columns 0..127, the gradient product at 128..255

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
  uint64_t bar[3];            // 0: the two partial copies, 1: first product, 2: second product
  long long ybase[8], xbase[8];
  int yrl[8], yrr[8], xrl[8], xrr[8];
  int item[8];
  uint32_t tmem;
  int valid, k, side, w;
};

struct GState {
  uint32_t tmem, bld, b1, b2, pld, p1, p2;
  bool pend1, pend2, pendld;
  int bad;
};

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 32 lanes x 8 consecutive FP32 columns
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// Shared-memory plan of a shape (RX, RY) for element size es: gM, R, one slice buffer and (BF16)
// the shared-memory copy of T.
__host__ __device__ constexpr uint32_t grad_slot(int es) { return 128u * 128u * (uint32_t)es; }
__host__ __device__ constexpr uint32_t grad_smem(int es, int RY) {
  return 2u * grad_slot(es) + 128u * (uint32_t)RY * (uint32_t)es + (es == 2 ? grad_slot(es) : 0u);
}

// One work item: the gradient of side `side` of a tile for core k. x0 / nx: the objects whose
// gradient is formed, y0 / ny: the others. Returns false (block-uniformly) on a timeout.
template <int KIND, int RX, int RY, typename ST>
__device__ bool grad_item(const GradTcArgs& g, char* sm, GState& st, GradShared& sh, int grp, int x0, int nx,
                          int y0, int ny, int side, int k, int d, const char* slots, float* outX) {
  using O = OpT<KIND>;
  constexpr int ES = O::ES, T = 16 / ES;
  constexpr int TX = 128 / RX, TY = 128 / RY;
  constexpr uint32_t SLOT = grad_slot(ES);
  constexpr uint32_t SBO = (128u / T) * 128u;          // full operand: bytes per 8 rows
  constexpr uint32_t SBOY = (uint32_t)(RY / T) * 128u;  // slice operand of one y: bytes per 8 rows
  constexpr uint32_t YSZ = (uint32_t)RY * RY * ES;     // bytes of one y's slice operand
  constexpr int KGY = RY / T, UPY = TY * RY * KGY / kGThreads, USY = kGThreads / RY;
  static_assert(UPY * kGThreads == TY * RY * KGY, "staging split");
  constexpr uint32_t ID1 = idesc(O::FMT, RY), ID2 = idesc(O::FMT, RX);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, h = warp >> 2;
  char* const mx = sm;
  char* const rg = sm + SLOT;
  char* const ysl = sm + 2 * SLOT;
  char* const ts = ysl + 128u * RY * ES;  // BF16 only
  const ST* const Yp = static_cast<const ST*>(g.mode == 0 ? (side ? g.A.p : g.B.p) : g.cores);
  const int sy = tid % RY, uy = tid / RY;

  // ---- the two partials: gM_k (slot k of the left sweep) and R_{k+1} (slot k of the right
  // sweep), in the orientation whose rows are this side's objects
  if (tid == 0) {
    expect_tx(st.bld, 2u * SLOT);
    bulk_g2s(su32(mx), slots + (size_t)(k * 2 + side) * SLOT, SLOT, st.bld);
    bulk_g2s(su32(rg), slots + (size_t)((d + k) * 2 + side) * SLOT, SLOT, st.bld);
  }
  st.pendld = true;
  // ---- objects of both sides at core k
  const int n = g.mode == 0 ? g.A.n[k] : g.nmodes[grp * g.dmax + k];
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

  // slice i of the y side -> registers: rows et' (right rank), K = et (left rank)
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
  auto store_slice = [&]() {
#pragma unroll
    for (int j = 0; j < UPY; ++j) {
      const int w = uy + j * USY, o = w / KGY, cg = w % KGY;
      const uint32_t off = (uint32_t)(sy >> 3) * SBOY + (uint32_t)cg * 128u + (uint32_t)(sy & 7) * 16u;
      *reinterpret_cast<uint4*>(ysl + o * YSZ + off) = pack_raw<KIND, ST, T>(py[j]);
    }
  };

  load_slice(0);
  st.bad |= !mbar_wait(st.bld, st.pld);
  st.pld ^= 1u;
  st.pendld = false;

  // lanes of this thread for the epilogue: row = (x, xi); this warp's quarter loads the columns
  // of the x blocks its 32 lanes cover, half h of them
  const int row = q * 32 + lane, xr = row / RX, xi = row % RX;
  constexpr int QCOLS = RX < 32 ? 32 : RX;   // columns of the blocks a lane quarter covers
  constexpr int HCOLS = QCOLS / 2;           // per column half
  const int cstart = ((q * 32) / RX) * RX + h * HCOLS;
  const bool xok = xr < nx && xi < sh.xrl[xr < 8 ? xr : 0];
  const int xrr = sh.xrr[xr < 8 ? xr : 0];
  const long long xrow = sh.xbase[xr < 8 ? xr : 0] + (long long)xi * n * xrr;

  for (int i = 0; i < n; ++i) {
    store_slice();
    async_fence();
    tc_before();
    if (__syncthreads_or(st.bad)) return false;
    // ---- first product: T for every y (columns y*RY ..)
    if (tid == 0) {
      tc_after();
#pragma unroll
      for (int y = 0; y < TY; ++y)
#pragma unroll
        for (int kk = 0; kk < RY / O::KI; ++kk) {
          const uint64_t da = sdesc2(su32(mx) + (uint32_t)((y * RY + kk * O::KI) / T) * 128u, 128u, SBO);
          const uint64_t db = sdesc2(su32(ysl) + (uint32_t)y * YSZ + (uint32_t)(kk * O::KI / T) * 128u, 128u, SBOY);
          mma<KIND>(st.tmem + (uint32_t)(y * RY), da, db, ID1, kk > 0 ? 1u : 0u);
        }
      mma_commit(st.b1);
    }
    st.pend1 = true;
    if (i + 1 < n) load_slice(i + 1);
    st.bad |= !mbar_wait(st.b1, st.p1);
    st.p1 ^= 1u;
    st.pend1 = false;
    tc_after();
    if constexpr (KIND == 1) {
      // T -> shared memory (rows (x, xi), K = (y, et')), rounded to BF16
#pragma unroll
      for (int cc = 0; cc < 64; cc += 16) {
        const int c0 = h * 64 + cc;
        float v[16];
        tmem_ld16(st.tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float u[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) u[t] = v[hh * 8 + t];
          *reinterpret_cast<uint4*>(ts + (uint32_t)(row >> 3) * SBO + (uint32_t)((c0 + hh * 8) / 8) * 128u +
                                    (uint32_t)(row & 7) * 16u) = O::pack(u);
        }
      }
      async_fence();
      tc_before();
      if (__syncthreads_or(st.bad)) return false;
    }
    // ---- second product: block x of (T R^T) for every x (columns 128 + x*RX ..), K = 128
    if (tid == 0) {
      tc_after();
#pragma unroll 1
      for (int x = 0; x < TX; ++x)
#pragma unroll
        for (int kk = 0; kk < 128 / O::KI; ++kk) {
          const uint64_t db =
              sdesc2(su32(rg) + (uint32_t)(x * RX / 8) * SBO + (uint32_t)(kk * O::KI / T) * 128u, 128u, SBO);
          if constexpr (KIND == 0) {
            mma_ts_tf32(st.tmem + 128u + (uint32_t)(x * RX), st.tmem + (uint32_t)(kk * O::KI), db, ID2, kk > 0 ? 1u : 0u);
          } else {
            const uint64_t da = sdesc2(su32(ts) + (uint32_t)(kk * O::KI / T) * 128u, 128u, SBO);
            mma<KIND>(st.tmem + 128u + (uint32_t)(x * RX), da, db, ID2, kk > 0 ? 1u : 0u);
          }
        }
      mma_commit(st.b2);
    }
    st.pend2 = true;
    st.bad |= !mbar_wait(st.b2, st.p2);
    st.p2 ^= 1u;
    st.pend2 = false;
    tc_after();
    // ---- epilogue: lane (x, xi) adds its block's columns to dX_x[xi, i, :]
#pragma unroll
    for (int cc = 0; cc < HCOLS; cc += 8) {
      const int c0 = cstart + cc;
      float v[8];
      tmem_ld8(st.tmem + 128u + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
      if (xok && outX) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = c0 + j, xc = c / RX, xp = c % RX;
          if (xc == xr && xp < xrr) atomicAdd(outX + xrow + (long long)i * xrr + xp, v[j]);
        }
      }
    }
  }
  return true;
}

__device__ __forceinline__ void grad_setup(GState& st, GradShared& sh, char* sm, uint32_t bytes) {
  const int tid = threadIdx.x, warp = tid >> 5;
  for (uint32_t e = (uint32_t)tid * 16u; e < bytes; e += kGThreads * 16u)
    *reinterpret_cast<uint4*>(sm + e) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0)
    for (int j = 0; j < 3; ++j) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sh.bar[j])));
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
  st.tmem = sh.tmem;
  st.bld = su32(&sh.bar[0]);
  st.b1 = su32(&sh.bar[1]);
  st.b2 = su32(&sh.bar[2]);
  st.pld = st.p1 = st.p2 = 0;
  st.pend1 = st.pend2 = st.pendld = false;
  st.bad = 0;
}

__device__ __forceinline__ void grad_teardown(const GradTcArgs& g, GState& st, bool failed) {
  if (failed) {
    // something did not signal completion: one more bounded wait for whatever is still in
    // flight (products and copies) before the tensor memory is released
    if (threadIdx.x == 0 && g.err) atomicExch(g.err, (int)T3F_ERR_TIMEOUT);
    if (st.pendld) mbar_wait(st.bld, st.pld);
    if (st.pend1) mbar_wait(st.b1, st.p1);
    if (st.pend2) mbar_wait(st.b2, st.p2);
  }
  tc_before();
  __syncthreads();
  tc_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(st.tmem), "r"(kGTmemCols));
}

template <int KIND, typename ST>
__device__ bool grad_dispatch(const GradTcArgs& g, char* sm, GState& st, GradShared& sh, int grp, int a0, int na,
                              int b0, int nb, int RA, int RB, int side, int k, int d, const char* slots, float* outX) {
  const int x0 = side ? b0 : a0, nx = side ? nb : na, y0 = side ? a0 : b0, ny = side ? na : nb;
  const int RX = side ? RB : RA, RY = side ? RA : RB;
  switch (RX * 1000 + RY) {
    case 16016: return grad_item<KIND, 16, 16, ST>(g, sm, st, sh, grp, x0, nx, y0, ny, side, k, d, slots, outX);
    case 16032: return grad_item<KIND, 16, 32, ST>(g, sm, st, sh, grp, x0, nx, y0, ny, side, k, d, slots, outX);
    case 16064: return grad_item<KIND, 16, 64, ST>(g, sm, st, sh, grp, x0, nx, y0, ny, side, k, d, slots, outX);
    case 32016: return grad_item<KIND, 32, 16, ST>(g, sm, st, sh, grp, x0, nx, y0, ny, side, k, d, slots, outX);
    case 32032: return grad_item<KIND, 32, 32, ST>(g, sm, st, sh, grp, x0, nx, y0, ny, side, k, d, slots, outX);
    case 32064: return grad_item<KIND, 32, 64, ST>(g, sm, st, sh, grp, x0, nx, y0, ny, side, k, d, slots, outX);
    case 64016: return grad_item<KIND, 64, 16, ST>(g, sm, st, sh, grp, x0, nx, y0, ny, side, k, d, slots, outX);
    case 64032: return grad_item<KIND, 64, 32, ST>(g, sm, st, sh, grp, x0, nx, y0, ny, side, k, d, slots, outX);
    default: return grad_item<KIND, 64, 64, ST>(g, sm, st, sh, grp, x0, nx, y0, ny, side, k, d, slots, outX);
  }
}

// Uniform batches: block = (tile, core, side); work list: persistent CTAs drain (tile, core,
// side) items through an atomic counter.
template <int KIND, typename ST>
__global__ void __launch_bounds__(kGThreads, 1) k_gram_tc_grad(const __grid_constant__ GradTcArgs g) {
  extern __shared__ __align__(128) char sm[];
  __shared__ __align__(16) GradShared sh;
  GState st;
  grad_setup(st, sh, sm, g.smem_bytes);
  constexpr uint32_t SLOT = grad_slot(OpT<KIND>::ES);
  const int tid = threadIdx.x;
  bool ok = true;
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
      ok = grad_dispatch<KIND, ST>(g, sm, st, sh, 0, a0, min(TA, g.A.batch - a0), b0, min(TB, g.B.batch - b0), RA, RB,
                                   side, k, d, slots, outX);
    }
  } else {
    while (ok) {
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
      ok = grad_dispatch<KIND, ST>(g, sm, st, sh, grp, a0, na, b0, nb, RA, RB, side, k, d, slots, g.dX);
    }
  }
  grad_teardown(g, st, !ok);
}

uint32_t grad_smem_max(int es) { return grad_smem(es, 64) + 1024u; }

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
