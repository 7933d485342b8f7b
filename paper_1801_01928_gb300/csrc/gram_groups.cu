// Pairwise Gram matrices within groups of a ragged collection of TT objects (uneven d, n
// and r; batches of the paper's Section 3.1, 'gram' and 'norm' of Section 4).
//
// Planning (host, t3f_gram_groups_prepare): the objects of every group are ordered by rank
// and split into rank buckets {<=8, <=16, <=32, <=64}; the upper triangle of each group's
// pairs is cut into tiles whose side depends on the buckets (tile table), the tiles are
// sorted by cost, largest first, and the work lists plus per-object tables are copied into
// the workspace once.
// Forward (t3f_gram_groups): one persistent launch of the tiled sweep kernel whose CTAs
// take tiles from the work list through an atomic counter, then the FP64 norms.
// Adjoint (t3f_gram_groups_backward): two persistent launches of the tiled adjoint kernel over
// work lists of smaller tiles (the adjoint keeps seven partial tiles in shared memory): tiles
// that need more than half an SM on 512-thread CTAs, one per SM, then the rest on 256-thread
// CTAs, two per SM; off-diagonal tiles use the symmetrised cotangent g_ab + g_ba. With a
// tensor-core math the sweeps over the tile list and the (tile, core, side) gradient items
// run instead. Every call only enqueues memsets and kernels, so it can be captured in a CUDA
// graph after one prepare.
#include <algorithm>
#include <math.h>
#include <vector>

#include "t3f_internal.cuh"

namespace t3f {

// kernels and helpers from gram_tile.cu / gram.cu
size_t gram_tile_smem(int TA, int TB, int RA, int RB);
t3f_status launch_gram_tile_table(const void* cores, int dtype, int dmax, const long long* off, const int* rk,
                                  const int* nmodes, const int* items, int nitems, int* head, const int* gstart,
                                  const int* gd, float* out, const long long* gout_off, const int* perm, size_t smem,
                                  cudaStream_t s);
size_t gram_tile_bwd_smem(int na, int nb, int RA, int RB, bool single);
bool gram_tile_bwd_fits(int na, int nb, int RA, int RB);
bool gram_tile_bwd_fits_small(int na, int nb, int RA, int RB, bool single);
t3f_status launch_gram_tile_bwd_table(const void* cores, int dtype, int dmax, const long long* off, const int* rk,
                                      const int* nmodes, const int* items, int nitems, int* head, const int* gstart,
                                      const int* gd, const int* perm, const float* dout, const long long* gout_off,
                                      float* dX, float* scratch, long long scratch_stride, size_t smem, int grid,
                                      int threads, cudaStream_t s);

t3f_status launch_gram_mma_list(int math, const void* cores, int dtype, int dmax, const long long* off,
                                const int* rk, const int* nmodes, const int* items, int nitems, int* head,
                                const int* gstart, const int* gd, float* gout, const long long* gout_off,
                                const int* perm, int* err, cudaStream_t s);
t3f_status launch_gram_tc_backward_list(int math, const void* cores, int dtype, int dmax, const long long* off,
                                        const int* rk, const int* nmodes, const int* items, int nitems,
                                        const int* gitems, int ngitems, int* heads, const int* gstart,
                                        const int* gd, const long long* gout_off, const int* perm,
                                        const float* dout, float* dX, char* scr, const long long* soff, int* err,
                                        cudaStream_t s);

namespace {

constexpr int kBuckets = 4;
constexpr int kMmaR[kBuckets] = {16, 16, 32, 64};  // tensor-core padded rank of each bucket
const int kBucketMax[kBuckets] = {8, 16, 32, 64};
const int kDefaultTiles[kBuckets] = {10, 6, 3, 1};

int sm_count_gg() { return device_sm_count(); }

struct Range {
  int begin, end, R;  // sorted positions [begin, end), padded inner rank
};

struct Plan {
  int count = 0, ngroups = 0, dmax = 0, nitems = 0;
  std::vector<int> sorted;   // sorted position -> object
  std::vector<int> perm;     // sorted position -> local index within the group
  std::vector<int> items;    // 8 ints per item (forward tiles, all bucket pairs)
  std::vector<int> mitems;   // tensor-core tiles (every bucket pair)
  int nmitems = 0;
  std::vector<long long> tsoff;  // tensor-core adjoint: first slot orientation of each tile
  std::vector<int> titems;   // tensor-core adjoint gradient items: tile, core, side, 0
  int ntitems = 0;
  long long tunits = 0;      // slot orientations (128 x 128 operands) of all tiles
  std::vector<int> bitems;   // 8 ints per item (adjoint tiles for 512-thread CTAs, one per SM)
  int nbitems = 0;
  size_t bsmem = 0;
  long long bstride = 0;     // scratch floats per CTA of the adjoint
  int bgrid = 0;
  std::vector<int> sitems;   // adjoint tiles for 256-thread CTAs, two per SM
  int nsitems = 0;
  size_t ssmem = 0;
  long long sstride = 0;
  int sgrid = 0;
  std::vector<long long> objoff;  // [pos][dmax]
  std::vector<int> objrk;    // [pos][dmax + 1]
  std::vector<int> nmodes;   // [group][dmax]
  std::vector<int> gd;       // [group]
  std::vector<int> gs;       // [group + 1]
  std::vector<long long> gout;  // [group]
  std::vector<Range> br;     // [group][bucket]
  size_t smem = 0;
  // workspace layout (bytes)
  size_t o_items, o_mitems, o_bitems, o_sitems, o_off, o_rk, o_nm, o_gs, o_gd, o_go, o_perm, o_scr, o_sscr, o_tsoff,
      o_titems, total;
};

int bucket_of(int r) {
  for (int b = 0; b < kBuckets; ++b)
    if (r <= kBucketMax[b]) return b;
  return -1;
}

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

t3f_status build_plan(const t3f_tt_ragged* X, int ngroups, const int* gstart, const int* tiles, Plan* P) {
  if (!X || !X->d || !X->n || !X->ranks || !X->obj_off || !X->cores) return T3F_ERR_ARG;
  if (X->count < 1 || ngroups < 1 || !gstart) return T3F_ERR_ARG;
  if (X->dtype != T3F_F32 && X->dtype != T3F_BF16) return T3F_ERR_DTYPE;
  if (gstart[0] != 0 || gstart[ngroups] != X->count) return T3F_ERR_SHAPE;
  int tl[kBuckets];
  for (int b = 0; b < kBuckets; ++b) {
    tl[b] = tiles ? tiles[b] : kDefaultTiles[b];
    if (tl[b] < 1 || tl[b] > 16) return T3F_ERR_ARG;
  }
  const int cnt = X->count;
  P->count = cnt;
  P->ngroups = ngroups;
  std::vector<int> noff(cnt + 1, 0), roff(cnt + 1, 0), rmax(cnt, 1);
  int dmax = 0;
  for (int o = 0; o < cnt; ++o) {
    const int d = X->d[o];
    if (d < 1 || d > T3F_MAX_D) return T3F_ERR_SHAPE;
    noff[o + 1] = noff[o] + d;
    roff[o + 1] = roff[o] + d + 1;
    dmax = std::max(dmax, d);
  }
  P->dmax = dmax;
  for (int o = 0; o < cnt; ++o) {
    const int d = X->d[o];
    const int* r = X->ranks + roff[o];
    if (r[0] != 1 || r[d] != 1) return T3F_ERR_SHAPE;
    for (int k = 0; k <= d; ++k) {
      if (r[k] < 1 || r[k] > T3F_MAX_RANK) return T3F_ERR_UNSUPPORTED;
      rmax[o] = std::max(rmax[o], r[k]);
    }
    for (int k = 0; k < d; ++k)
      if (X->n[noff[o] + k] < 1 || X->n[noff[o] + k] > T3F_MAX_MODE) return T3F_ERR_SHAPE;
  }
  P->gs.assign(gstart, gstart + ngroups + 1);
  P->gd.resize(ngroups);
  P->nmodes.assign((size_t)ngroups * dmax, 1);
  P->gout.resize(ngroups);
  long long go = 0;
  for (int g = 0; g < ngroups; ++g) {
    if (gstart[g + 1] <= gstart[g]) return T3F_ERR_SHAPE;
    const int o0 = gstart[g];
    P->gd[g] = X->d[o0];
    for (int o = o0; o < gstart[g + 1]; ++o) {
      if (X->d[o] != P->gd[g]) return T3F_ERR_SHAPE;
      for (int k = 0; k < P->gd[g]; ++k)
        if (X->n[noff[o] + k] != X->n[noff[o0] + k]) return T3F_ERR_SHAPE;
    }
    for (int k = 0; k < P->gd[g]; ++k) P->nmodes[(size_t)g * dmax + k] = X->n[noff[o0] + k];
    P->gout[g] = go;
    const long long S = gstart[g + 1] - gstart[g];
    go += S * S;
  }
  // order every group by rank (stable) and record the bucket ranges
  P->sorted.resize(cnt);
  P->perm.resize(cnt);
  P->br.assign((size_t)ngroups * kBuckets, Range{0, 0, 0});
  for (int g = 0; g < ngroups; ++g) {
    std::vector<int> ids;
    for (int o = gstart[g]; o < gstart[g + 1]; ++o) ids.push_back(o);
    std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) { return rmax[x] < rmax[y]; });
    for (size_t q = 0; q < ids.size(); ++q) {
      P->sorted[gstart[g] + q] = ids[q];
      P->perm[gstart[g] + q] = ids[q] - gstart[g];
    }
    int pos = gstart[g];
    for (int b = 0; b < kBuckets; ++b) {
      Range r{pos, pos, 0};
      while (pos < gstart[g + 1] && bucket_of(rmax[P->sorted[pos]]) == b) {
        r.R = std::max(r.R, rmax[P->sorted[pos]]);
        ++pos;
      }
      r.end = pos;
      r.R = (r.R + 3) & ~3;
      P->br[(size_t)g * kBuckets + b] = r;
    }
  }
  // per-object tables in sorted order
  P->objoff.assign((size_t)cnt * dmax, 0);
  P->objrk.assign((size_t)cnt * (dmax + 1), 1);
  for (int pos = 0; pos < cnt; ++pos) {
    const int o = P->sorted[pos];
    const int d = X->d[o];
    long long off = X->obj_off[o];
    for (int k = 0; k < d; ++k) {
      const int r0 = X->ranks[roff[o] + k], r1 = X->ranks[roff[o] + k + 1], n = X->n[noff[o] + k];
      P->objoff[(size_t)pos * dmax + k] = off;
      off += (long long)r0 * n * r1;
    }
    for (int k = 0; k <= d; ++k) P->objrk[(size_t)pos * (dmax + 1) + k] = X->ranks[roff[o] + k];
  }
  // CUDA-core tiles of the upper triangle of every group, cut per bucket pair from the
  // objects' own padded ranks: a run of consecutive objects (sorted by rank) grows up to the
  // side cap while its square self-tile fits one CTA, so the lower-rank runs of a bucket get
  // more pairs per CTA; a cross tile of two runs that does not fit is halved along b until
  // it does. A tile that is a sub-tile of a diagonal square covers ordered pairs (sym = 0).
  auto padr = [&](int pos0, int n) {
    int R = 4;
    for (int x = pos0; x < pos0 + n; ++x) R = std::max(R, (rmax[P->sorted[x]] + 3) & ~3);
    return R;
  };
  auto make_items = [&](const int* cap, std::vector<int>* out, size_t* smem_out, long long* pmax_out) -> t3f_status {
    // a tile must fit one CTA of 512 threads: at most 2 blocks each, staging and shared memory
    auto tile_ok = [&](int na, int nb, int RA, int RB) {
      if (na * (RA / 4) * nb * (RB / 4) > 1024) return false;
      return gram_tile_smem(na, nb, RA, RB) <= 200 * 1024 && na * RA * RA + nb * RB * RB <= 512 * 16;
    };
    auto cut = [&](const Range& Rg, int side_max, std::vector<std::pair<int, int>>* runs) {
      for (int s0 = Rg.begin; s0 < Rg.end;) {
        int n = 1;
        while (n < side_max && s0 + n < Rg.end) {
          const int R = padr(s0, n + 1);
          if (!tile_ok(n + 1, n + 1, R, R)) break;
          ++n;
        }
        runs->push_back({s0, n});
        s0 += n;
      }
    };
    struct It {
      double cost;
      int v[8];
    };
    std::vector<It> its;
    size_t smem = 0;
    long long pmax = 0;
    for (int g = 0; g < ngroups; ++g) {
      double slices = 0;
      for (int k = 0; k < P->gd[g]; ++k) slices += P->nmodes[(size_t)g * dmax + k];
      for (int p = 0; p < kBuckets; ++p)
        for (int q = p; q < kBuckets; ++q) {
          const Range& A = P->br[(size_t)g * kBuckets + p];
          const Range& B = P->br[(size_t)g * kBuckets + q];
          if (A.end == A.begin || B.end == B.begin) continue;
          std::vector<std::pair<int, int>> ta, tb;
          cut(A, cap[p], &ta);
          cut(B, cap[q], &tb);
          for (size_t ia = 0; ia < ta.size(); ++ia) {
            const int a0 = ta[ia].first, na = ta[ia].second, RA = padr(a0, na);
            // same bucket: the b runs start at the a run, the diagonal tile covers its square
            for (size_t ib = (p == q ? ia : 0); ib < tb.size(); ++ib) {
              int sym = (p == q && ib == ia) ? 0 : 1;
              std::pair<int, int> brun = tb[ib];
              bool merged = false;
              // single objects on both sides (high ranks, where no 2 x 2 square fits): a 1 x 1
              // tile fills at most half of the CTA's threads, so two neighbouring single b runs
              // form one 1 x 2 tile when its blocks and shared memory fit (the staging loop
              // takes any number of rows per thread). The tile writes both G_ab and G_ba
              // (sym = 1); an object's pair with itself may be the first of the two, its entry
              // is then written twice with the same value.
              if (na == 1 && brun.second == 1 && ib + 1 < tb.size() && tb[ib + 1].second == 1 &&
                  (RA / 4) * 2 * (padr(brun.first, 2) / 4) <= 1024 &&
                  gram_tile_smem(1, 2, RA, padr(brun.first, 2)) <= 200 * 1024) {
                brun.second = 2;
                merged = true;
                sym = 1;
                ++ib;
              }
              std::vector<std::pair<int, int>> todo{brun};
              while (!todo.empty()) {
                const int b0 = todo.back().first, nb = todo.back().second;
                todo.pop_back();
                const int RB = padr(b0, nb);
                if (!(merged && nb == 2) && !tile_ok(na, nb, RA, RB)) {
                  if (nb == 1) return T3F_ERR_UNSUPPORTED;
                  todo.push_back({b0 + nb / 2, nb - nb / 2});
                  todo.push_back({b0, nb / 2});
                  continue;
                }
                It it;
                it.cost = (double)na * nb * RA * RB * (RA + RB) * slices;
                it.v[0] = g;
                it.v[1] = a0;
                it.v[2] = na;
                it.v[3] = b0;
                it.v[4] = nb;
                it.v[5] = RA;
                it.v[6] = RB;
                it.v[7] = sym;
                its.push_back(it);
                smem = std::max(smem, gram_tile_smem(na, nb, RA, RB));
                pmax = std::max(pmax, (long long)na * nb * RA * RB);
              }
            }
          }
        }
    }
    std::stable_sort(its.begin(), its.end(), [](const It& x, const It& y) { return x.cost > y.cost; });
    out->resize(its.size() * 8);
    for (size_t w = 0; w < its.size(); ++w)
      for (int q = 0; q < 8; ++q) (*out)[w * 8 + q] = its[w].v[q];
    *smem_out = smem;
    *pmax_out = pmax;
    return T3F_OK;
  };
  size_t smem = 0;
  long long pmax = 0;
  T3F_CHECK(make_items(tl, &P->items, &smem, &pmax));
  P->nitems = (int)(P->items.size() / 8);
  // tensor-core tiles for every bucket pair p <= q: the a side pads to RA = 16 / 16 / 32 / 64
  // (bucket p), the b side to RB (bucket q); (128 / RA) x (128 / RB) pairs per tile
  {
    struct It {
      double cost;
      int v[8];
    };
    std::vector<It> its;
    for (int g = 0; g < ngroups; ++g) {
      double slices = 0;
      for (int k = 0; k < P->gd[g]; ++k) slices += P->nmodes[(size_t)g * dmax + k];
      for (int p = 0; p < kBuckets; ++p)
        for (int q = p; q < kBuckets; ++q) {
          const Range& A = P->br[(size_t)g * kBuckets + p];
          const Range& B = P->br[(size_t)g * kBuckets + q];
          if (A.end == A.begin || B.end == B.begin) continue;
          const int RA = kMmaR[p], RB = kMmaR[q], TA = 128 / RA, TB = 128 / RB;
          for (int a0 = A.begin; a0 < A.end; a0 += TA) {
            const int na = std::min(TA, A.end - a0);
            // same bucket: b tiles start at the a tile's first object so the pairs below the
            // diagonal are covered once through the symmetric write
            for (int b0 = (p == q ? a0 : B.begin); b0 < B.end; b0 += TB) {
              const int nb = std::min(TB, B.end - b0);
              It it;
              it.cost = 128.0 * 128.0 * (RA + RB) * slices;
              it.v[0] = g;
              it.v[1] = a0;
              it.v[2] = na;
              it.v[3] = b0;
              it.v[4] = nb;
              it.v[5] = RA;
              it.v[6] = (p == q && a0 == b0) ? 0 : 1;
              it.v[7] = RB;
              its.push_back(it);
            }
          }
        }
    }
    // grouped by tile shape (largest first), then by cost: a CTA rarely switches between the
    // shapes' code paths, which keeps the instruction cache warm
    std::stable_sort(its.begin(), its.end(), [](const It& x, const It& y) {
      if (x.v[7] != y.v[7]) return x.v[7] > y.v[7];
      if (x.v[5] != y.v[5]) return x.v[5] > y.v[5];
      return x.cost > y.cost;
    });
    P->mitems.resize(its.size() * 8);
    for (size_t w = 0; w < its.size(); ++w)
      for (int x = 0; x < 8; ++x) P->mitems[w * 8 + x] = its[w].v[x];
    P->nmitems = (int)its.size();
    // tensor-core adjoint: every tile keeps both sweep directions' partials (d interfaces
    // each, two orientations); one gradient item per (tile, core, side), largest first
    struct Gi {
      double cost;
      int v[4];
    };
    std::vector<Gi> gis;
    long long u = 0;
    P->tsoff.resize(its.size());
    for (size_t w = 0; w < its.size(); ++w) {
      const int g = its[w].v[0], d = P->gd[g], RA = its[w].v[5], RB = its[w].v[7];
      P->tsoff[w] = u;
      u += 4LL * d;
      for (int k = 0; k < d; ++k)
        for (int side = 0; side < 2; ++side) {
          Gi gi;
          gi.cost = (double)P->nmodes[(size_t)g * dmax + k] * (128.0 + (side ? RA : RB));
          gi.v[0] = (int)w;
          gi.v[1] = k;
          gi.v[2] = side;
          gi.v[3] = 0;
          gis.push_back(gi);
        }
    }
    std::stable_sort(gis.begin(), gis.end(), [](const Gi& x, const Gi& y) { return x.cost > y.cost; });
    P->titems.resize(gis.size() * 4);
    for (size_t w = 0; w < gis.size(); ++w)
      for (int x = 0; x < 4; ++x) P->titems[w * 4 + x] = gis[w].v[x];
    P->ntitems = (int)gis.size();
    P->tunits = u;
  }
  // adjoint tiles (seven partial tiles per pair). Runs of rank-sorted objects grow (side at
  // most 16) while their square tile fits a full-size CTA (512 threads, one per SM); a tile
  // that does not fit is halved along b, then along a. Tiles that also fit a half-size CTA
  // (256 threads, half an SM's shared memory), if need be with one staging buffer instead of
  // two, go to a second list run with two CTAs per SM, where one CTA's barrier and load waits
  // overlap the other's work. Sub-tiles of a diagonal square cover ordered pairs (sym = 0).
  {
    auto padr = [&](int pos0, int n) {
      int R = 4;
      for (int x = pos0; x < pos0 + n; ++x) R = std::max(R, (rmax[P->sorted[x]] + 3) & ~3);
      return R;
    };
    // full-size tiles: one 4 x 4 block per thread of 512 (the kernel's one-block form)
    auto fits_big = [&](int na, int nb, int RA, int RB) {
      return na * (RA / 4) * nb * (RB / 4) <= 512 && gram_tile_bwd_fits(na, nb, RA, RB);
    };
    struct It {
      double cost;
      int v[8];
    };
    std::vector<It> big, small;
    size_t bsm = 0, ssm = 0;
    long long bpm = 0, spm = 0;
    for (int g = 0; g < ngroups; ++g) {
      double slices = 0;
      for (int k = 0; k < P->gd[g]; ++k) slices += P->nmodes[(size_t)g * dmax + k];
      auto cut = [&](const Range& Rg, std::vector<std::pair<int, int>>* runs) {
        for (int s0 = Rg.begin; s0 < Rg.end;) {
          int n = 1;
          while (n < 16 && s0 + n < Rg.end) {
            const int R = padr(s0, n + 1);
            if (!fits_big(n + 1, n + 1, R, R)) break;
            ++n;
          }
          runs->push_back({s0, n});
          s0 += n;
        }
      };
      for (int p = 0; p < kBuckets; ++p)
        for (int q = p; q < kBuckets; ++q) {
          const Range& A = P->br[(size_t)g * kBuckets + p];
          const Range& B = P->br[(size_t)g * kBuckets + q];
          if (A.end == A.begin || B.end == B.begin) continue;
          std::vector<std::pair<int, int>> ta, tb;
          cut(A, &ta);
          cut(B, &tb);
          for (size_t ia = 0; ia < ta.size(); ++ia)
            for (size_t ib = (p == q ? ia : 0); ib < tb.size(); ++ib) {
              const int sym = (p == q && ib == ia) ? 0 : 1;
              struct Tl {
                int a0, na, b0, nb;
              };
              std::vector<Tl> todo{{ta[ia].first, ta[ia].second, tb[ib].first, tb[ib].second}};
              while (!todo.empty()) {
                const Tl t = todo.back();
                todo.pop_back();
                const int RA = padr(t.a0, t.na), RB = padr(t.b0, t.nb);
                const bool fb = fits_big(t.na, t.nb, RA, RB);
                if (!fb && t.nb > 1) {
                  todo.push_back({t.a0, t.na, t.b0 + t.nb / 2, t.nb - t.nb / 2});
                  todo.push_back({t.a0, t.na, t.b0, t.nb / 2});
                  continue;
                }
                if (!fb && t.na > 1) {
                  todo.push_back({t.a0 + t.na / 2, t.na - t.na / 2, t.b0, t.nb});
                  todo.push_back({t.a0, t.na / 2, t.b0, t.nb});
                  continue;
                }
                if (!fb) return T3F_ERR_UNSUPPORTED;
                // half-size CTA with two staging buffers, else with one, else full-size
                const bool fs2 = gram_tile_bwd_fits_small(t.na, t.nb, RA, RB, false);
                const bool fs = fs2 || gram_tile_bwd_fits_small(t.na, t.nb, RA, RB, true);
                It it;
                it.cost = (double)t.na * t.nb * RA * RB * (3.0 * RA + 4.0 * RB) * slices;
                it.v[0] = g;
                it.v[1] = t.a0;
                it.v[2] = t.na;
                it.v[3] = t.b0;
                it.v[4] = t.nb;
                it.v[5] = RA;
                it.v[6] = RB;
                it.v[7] = sym | (fs && !fs2 ? 2 : 0);  // bit 1: one staging buffer
                const size_t sm = gram_tile_bwd_smem(t.na, t.nb, RA, RB, fs && !fs2);
                const long long pe = (long long)t.na * t.nb * RA * RB;
                if (fs) {
                  small.push_back(it);
                  ssm = std::max(ssm, sm);
                  spm = std::max(spm, pe);
                } else {
                  big.push_back(it);
                  bsm = std::max(bsm, sm);
                  bpm = std::max(bpm, pe);
                }
              }
            }
        }
    }
    auto flat = [](std::vector<It>& its, std::vector<int>* out) {
      std::stable_sort(its.begin(), its.end(), [](const It& x, const It& y) { return x.cost > y.cost; });
      out->resize(its.size() * 8);
      for (size_t w = 0; w < its.size(); ++w)
        for (int q = 0; q < 8; ++q) (*out)[w * 8 + q] = its[w].v[q];
    };
    flat(big, &P->bitems);
    flat(small, &P->sitems);
    P->nbitems = (int)big.size();
    P->bsmem = bsm;
    P->bstride = (long long)(dmax + 1) * bpm;
    P->bgrid = std::max(1, std::min(P->nbitems, sm_count_gg()));
    P->nsitems = (int)small.size();
    P->ssmem = ssm;
    P->sstride = (long long)(dmax + 1) * spm;
    P->sgrid = std::max(1, std::min(P->nsitems, 2 * sm_count_gg()));
  }
  P->smem = smem;
  size_t o = kWsHeader;
  P->o_items = o; o += a256(sizeof(int) * P->items.size());
  P->o_mitems = o; o += a256(sizeof(int) * P->mitems.size());
  P->o_bitems = o; o += a256(sizeof(int) * P->bitems.size());
  P->o_sitems = o; o += a256(sizeof(int) * P->sitems.size());
  P->o_off = o; o += a256(sizeof(long long) * P->objoff.size());
  P->o_rk = o; o += a256(sizeof(int) * P->objrk.size());
  P->o_nm = o; o += a256(sizeof(int) * P->nmodes.size());
  P->o_gs = o; o += a256(sizeof(int) * P->gs.size());
  P->o_gd = o; o += a256(sizeof(int) * P->gd.size());
  P->o_go = o; o += a256(sizeof(long long) * P->gout.size());
  P->o_perm = o; o += a256(sizeof(int) * P->perm.size());
  P->o_scr = o; o += a256(sizeof(float) * (size_t)P->bstride * P->bgrid);
  P->o_sscr = o; o += a256(sizeof(float) * (size_t)P->sstride * P->sgrid);
  P->o_tsoff = o; o += a256(sizeof(long long) * P->tsoff.size());
  P->o_titems = o; o += a256(sizeof(int) * P->titems.size());
  P->total = o;
  return T3F_OK;
}

// ---------------------------------------------------------------------------------------
// small kernels: FP64 norms, pack / unpack of padded batches, cotangent gather
// ---------------------------------------------------------------------------------------

__global__ void k_group_norms(const float* out, const long long* gout_off, const int* gs, int ngroups, double* norms) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < gs[ngroups]; o += gridDim.x * blockDim.x) {
    int g = 0;
    while (gs[g + 1] <= o) ++g;
    const int S = gs[g + 1] - gs[g], l = o - gs[g];
    norms[o] = sqrt(fmax((double)out[gout_off[g] + (long long)l * S + l], 0.0));
  }
}

}  // namespace

t3f_status gg_tables_upload(const Plan& P, char* w, cudaStream_t s) {
  struct Cp {
    size_t off;
    const void* src;
    size_t bytes;
  } cps[] = {{P.o_items, P.items.data(), sizeof(int) * P.items.size()},
             {P.o_mitems, P.mitems.data(), sizeof(int) * P.mitems.size()},
             {P.o_bitems, P.bitems.data(), sizeof(int) * P.bitems.size()},
             {P.o_sitems, P.sitems.data(), sizeof(int) * P.sitems.size()},
             {P.o_off, P.objoff.data(), sizeof(long long) * P.objoff.size()},
             {P.o_rk, P.objrk.data(), sizeof(int) * P.objrk.size()},
             {P.o_nm, P.nmodes.data(), sizeof(int) * P.nmodes.size()},
             {P.o_gs, P.gs.data(), sizeof(int) * P.gs.size()},
             {P.o_gd, P.gd.data(), sizeof(int) * P.gd.size()},
             {P.o_go, P.gout.data(), sizeof(long long) * P.gout.size()},
             {P.o_perm, P.perm.data(), sizeof(int) * P.perm.size()},
             {P.o_tsoff, P.tsoff.data(), sizeof(long long) * P.tsoff.size()},
             {P.o_titems, P.titems.data(), sizeof(int) * P.titems.size()}};
  for (const Cp& c : cps)
    if (c.bytes && cudaMemcpyAsync(w + c.off, c.src, c.bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return T3F_ERR_CUDA;
  return T3F_OK;
}

}  // namespace t3f

using namespace t3f;

extern "C" size_t t3f_gram_groups_workspace_size(const t3f_tt_ragged* X, int32_t ngroups, const int32_t* gstart,
                                                 const int32_t* tiles) {
  Plan P;
  if (build_plan(X, ngroups, gstart, tiles, &P) != T3F_OK) return 0;
  return P.total;
}

// Scratch of the tensor-core adjoint: every slot orientation is a 128 x 128 operand of the
// math's element type.
size_t gg_tc_scratch(const Plan& P, int math) {
  const size_t es = math == T3F_MATH_TF32 ? 4 : 2;
  return (size_t)P.tunits * 128u * 128u * es;
}

extern "C" size_t t3f_gram_groups_backward_workspace_size(const t3f_tt_ragged* X, int32_t ngroups,
                                                          const int32_t* gstart, const int32_t* tiles,
                                                          int32_t math) {
  Plan P;
  if (build_plan(X, ngroups, gstart, tiles, &P) != T3F_OK) return 0;
  if (math == T3F_MATH_FP32) return P.total;
  if (math != T3F_MATH_TF32 && math != T3F_MATH_BF16) return 0;
  return P.total + gg_tc_scratch(P, math);
}

extern "C" t3f_status t3f_gram_groups_prepare(const t3f_tt_ragged* X, int32_t ngroups, const int32_t* gstart,
                                              const int32_t* tiles, void* ws, size_t ws_bytes, t3f_stream_t stream) {
  Plan P;
  T3F_CHECK(build_plan(X, ngroups, gstart, tiles, &P));
  T3F_CHECK(check_ws(ws, ws_bytes, P.total));
  return gg_tables_upload(P, static_cast<char*>(ws), (cudaStream_t)stream);
}

extern "C" t3f_status t3f_gram_groups(const t3f_tt_ragged* X, int32_t ngroups, const int32_t* gstart,
                                      const int32_t* tiles, int32_t math, float* out, double* norms, void* ws,
                                      size_t ws_bytes, t3f_stream_t stream) {
  Plan P;
  T3F_CHECK(build_plan(X, ngroups, gstart, tiles, &P));
  T3F_CHECK(check_ws(ws, ws_bytes, P.total));
  if (!out) return T3F_ERR_ARG;
  if (math != T3F_MATH_FP32 && math != T3F_MATH_TF32 && math != T3F_MATH_BF16) return T3F_ERR_ARG;
  if (math == T3F_MATH_TF32 && X->dtype != T3F_F32) return T3F_ERR_DTYPE;
  cudaStream_t s = (cudaStream_t)stream;
  char* w = static_cast<char*>(ws);
  // header words: 0 error, 1 CUDA-core list head, 3 tensor-core list head (2 and 4: the
  // adjoint lists)
  int* hw = reinterpret_cast<int*>(w);
  if (cudaMemsetAsync(w, 0, 8 * sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
  const long long* off = reinterpret_cast<const long long*>(w + P.o_off);
  const int* rk = reinterpret_cast<const int*>(w + P.o_rk);
  const int* nm = reinterpret_cast<const int*>(w + P.o_nm);
  const int* gsd = reinterpret_cast<const int*>(w + P.o_gs);
  const int* gdd = reinterpret_cast<const int*>(w + P.o_gd);
  const long long* god = reinterpret_cast<const long long*>(w + P.o_go);
  const int* pd = reinterpret_cast<const int*>(w + P.o_perm);
  if (math == T3F_MATH_FP32) {
    T3F_CHECK(launch_gram_tile_table(X->cores, X->dtype, P.dmax, off, rk, nm,
                                     reinterpret_cast<const int*>(w + P.o_items), P.nitems, hw + 1, gsd, gdd, out,
                                     god, pd, P.smem, s));
  } else {
    if (P.nmitems > 0)
      T3F_CHECK(launch_gram_mma_list(math, X->cores, X->dtype, P.dmax, off, rk, nm,
                                     reinterpret_cast<const int*>(w + P.o_mitems), P.nmitems, hw + 3, gsd, gdd, out,
                                     god, pd, hw, s));
  }
  if (norms) {
    k_group_norms<<<(P.count + 255) / 256, 256, 0, s>>>(out, reinterpret_cast<const long long*>(w + P.o_go),
                                                         reinterpret_cast<const int*>(w + P.o_gs), ngroups, norms);
    T3F_CHECK(launch_status());
  }
  return T3F_OK;
}

extern "C" t3f_status t3f_gram_groups_backward(const t3f_tt_ragged* X, int32_t ngroups, const int32_t* gstart,
                                               const int32_t* tiles, int32_t math, const float* dout, float* dcores,
                                               void* ws, size_t ws_bytes, t3f_stream_t stream) {
  Plan P;
  T3F_CHECK(build_plan(X, ngroups, gstart, tiles, &P));
  if (math != T3F_MATH_FP32 && math != T3F_MATH_TF32 && math != T3F_MATH_BF16) return T3F_ERR_ARG;
  if (math == T3F_MATH_TF32 && X->dtype != T3F_F32) return T3F_ERR_DTYPE;
  T3F_CHECK(check_ws(ws, ws_bytes, P.total + (math == T3F_MATH_FP32 ? 0 : gg_tc_scratch(P, math))));
  if (!dout || !dcores) return T3F_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  char* w = static_cast<char*>(ws);
  long long nel = 0;  // elements of the ragged cores
  {
    long long no = 0, ro = 0;
    for (int o = 0; o < X->count; ++o) {
      long long e = 0;
      for (int k = 0; k < X->d[o]; ++k) e += (long long)X->ranks[ro + k] * X->n[no + k] * X->ranks[ro + k + 1];
      nel = std::max(nel, X->obj_off[o] + e);
      no += X->d[o];
      ro += X->d[o] + 1;
    }
  }
  if (cudaMemsetAsync(dcores, 0, sizeof(float) * nel, s) != cudaSuccess) return T3F_ERR_CUDA;
  if (math != T3F_MATH_FP32) {
    // header words: 0 error, 5 and 6 the sweep and gradient list heads
    int* hw = reinterpret_cast<int*>(w);
    if (cudaMemsetAsync(hw, 0, sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
    if (cudaMemsetAsync(hw + 5, 0, 2 * sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
    return launch_gram_tc_backward_list(
        math, X->cores, X->dtype, P.dmax, reinterpret_cast<const long long*>(w + P.o_off),
        reinterpret_cast<const int*>(w + P.o_rk), reinterpret_cast<const int*>(w + P.o_nm),
        reinterpret_cast<const int*>(w + P.o_mitems), P.nmitems, reinterpret_cast<const int*>(w + P.o_titems),
        P.ntitems, hw + 5, reinterpret_cast<const int*>(w + P.o_gs), reinterpret_cast<const int*>(w + P.o_gd),
        reinterpret_cast<const long long*>(w + P.o_go), reinterpret_cast<const int*>(w + P.o_perm), dout, dcores,
        w + P.total, reinterpret_cast<const long long*>(w + P.o_tsoff), hw, s);
  }
  // list heads: header word 2 (full-size CTAs) and word 4 (half-size CTAs)
  int* head = reinterpret_cast<int*>(w + 2 * sizeof(int));
  int* shead = reinterpret_cast<int*>(w + 4 * sizeof(int));
  if (cudaMemsetAsync(head, 0, sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
  if (cudaMemsetAsync(shead, 0, sizeof(int), s) != cudaSuccess) return T3F_ERR_CUDA;
  // the full-size list first (its items are the most expensive), then the half-size one
  if (P.nbitems > 0)
    T3F_CHECK(launch_gram_tile_bwd_table(
        X->cores, X->dtype, P.dmax, reinterpret_cast<const long long*>(w + P.o_off),
        reinterpret_cast<const int*>(w + P.o_rk), reinterpret_cast<const int*>(w + P.o_nm),
        reinterpret_cast<const int*>(w + P.o_bitems), P.nbitems, head, reinterpret_cast<const int*>(w + P.o_gs),
        reinterpret_cast<const int*>(w + P.o_gd), reinterpret_cast<const int*>(w + P.o_perm), dout,
        reinterpret_cast<const long long*>(w + P.o_go), dcores, reinterpret_cast<float*>(w + P.o_scr), P.bstride,
        P.bsmem, P.bgrid, 512, s));
  if (P.nsitems > 0)
    T3F_CHECK(launch_gram_tile_bwd_table(
        X->cores, X->dtype, P.dmax, reinterpret_cast<const long long*>(w + P.o_off),
        reinterpret_cast<const int*>(w + P.o_rk), reinterpret_cast<const int*>(w + P.o_nm),
        reinterpret_cast<const int*>(w + P.o_sitems), P.nsitems, shead, reinterpret_cast<const int*>(w + P.o_gs),
        reinterpret_cast<const int*>(w + P.o_gd), reinterpret_cast<const int*>(w + P.o_perm), dout,
        reinterpret_cast<const long long*>(w + P.o_go), dcores, reinterpret_cast<float*>(w + P.o_sscr), P.sstride,
        P.ssmem, P.sgrid, 256, s));
  return T3F_OK;
}
