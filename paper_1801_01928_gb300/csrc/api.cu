// Descriptor validation, status strings and small host-only entry points of libt3f.
#include <string.h>

#include <atomic>

#include "t3f_internal.cuh"

namespace t3f {

t3f_status make_view(const t3f_tt* t, TTV* v, int want_dtype, bool matrix_expected) {
  if (!t || !v) return T3F_ERR_ARG;
  if (t->d < 1 || t->d > T3F_MAX_D || t->batch < 1) return T3F_ERR_ARG;
  if (!t->n || !t->ranks || !t->cores) return T3F_ERR_ARG;
  if (t->dtype != T3F_F32 && t->dtype != T3F_F64 && t->dtype != T3F_BF16) return T3F_ERR_ARG;
  if (want_dtype >= 0 && t->dtype != want_dtype) return T3F_ERR_DTYPE;
  if (matrix_expected != (t->m != nullptr)) return T3F_ERR_SHAPE;
  memset(v, 0, sizeof(*v));
  v->d = t->d;
  v->batch = t->batch;
  v->dtype = t->dtype;
  v->is_matrix = t->m != nullptr;
  v->p = t->cores;
  if (t->ranks[0] != 1 || t->ranks[t->d] != 1) return T3F_ERR_SHAPE;
  long long off = 0;
  for (int k = 0; k <= t->d; ++k) {
    if (t->ranks[k] < 1 || t->ranks[k] > (1 << 20)) return T3F_ERR_SHAPE;
    v->r[k] = t->ranks[k];
    v->rmax = v->r[k] > v->rmax ? v->r[k] : v->rmax;
  }
  for (int k = 0; k < t->d; ++k) {
    int nk = t->n[k];
    int mk = t->m ? t->m[k] : 1;
    if (nk < 1 || nk > T3F_MAX_MODE || mk < 1 || mk > T3F_MAX_MODE) return T3F_ERR_SHAPE;
    v->n[k] = nk;
    v->m[k] = mk;
    v->nmax = nk > v->nmax ? nk : v->nmax;
    long long sz = (long long)v->r[k] * mk * nk * v->r[k + 1];
    if (sz > (1LL << 40) / t->batch) return T3F_ERR_SHAPE;
    v->osz[k] = sz;
    v->off[k] = off;
    off += sz * t->batch;
  }
  return T3F_OK;
}

t3f_status check_ws(void* ws, size_t ws_bytes, size_t need) {
  if (need == 0) return T3F_OK;
  if (!ws || ws_bytes < need) return T3F_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return T3F_ERR_WORKSPACE;
  return T3F_OK;
}

static std::atomic<long long> g_launches{0};

t3f_status launch_status() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? T3F_OK : T3F_ERR_CUDA;
}

}  // namespace t3f

using namespace t3f;

extern "C" const char* t3f_status_string(int32_t status) {
  switch (status) {
    case T3F_OK: return "T3F_OK";
    case T3F_ERR_ARG: return "T3F_ERR_ARG: invalid argument";
    case T3F_ERR_SHAPE: return "T3F_ERR_SHAPE: operand shapes disagree";
    case T3F_ERR_DTYPE: return "T3F_ERR_DTYPE: unsupported storage type";
    case T3F_ERR_WORKSPACE: return "T3F_ERR_WORKSPACE: workspace too small or misaligned";
    case T3F_ERR_CUDA: return "T3F_ERR_CUDA: CUDA launch/runtime error";
    case T3F_ERR_TIMEOUT: return "T3F_ERR_TIMEOUT: bounded device wait ran out";
    case T3F_ERR_UNSUPPORTED: return "T3F_ERR_UNSUPPORTED: beyond this build's kernel limits";
    default: return "unknown t3f status";
  }
}

extern "C" int32_t t3f_version(void) { return 100; }

extern "C" int64_t t3f_packed_size(const t3f_tt* t) {
  TTV v;
  if (!t) return 0;
  if (make_view(t, &v, -1, t->m != nullptr) != T3F_OK) return 0;
  long long tot = 0;
  for (int k = 0; k < v.d; ++k) tot += v.osz[k] * v.batch;
  return tot;
}

extern "C" t3f_status t3f_orth_ranks(int32_t d, const int32_t* n, const int32_t* ranks,
                                     int32_t* out_ranks) {
  if (d < 1 || d > T3F_MAX_D || !n || !ranks || !out_ranks) return T3F_ERR_ARG;
  if (ranks[0] != 1 || ranks[d] != 1) return T3F_ERR_SHAPE;
  long long r1[T3F_MAX_D + 1];
  for (int k = 0; k <= d; ++k) {
    if (ranks[k] < 1) return T3F_ERR_SHAPE;
    r1[k] = ranks[k];
  }
  for (int k = 0; k < d; ++k)
    if (n[k] < 1) return T3F_ERR_SHAPE;
  for (int k = d - 1; k >= 1; --k) {
    long long c = (long long)n[k] * r1[k + 1];
    if (c < r1[k]) r1[k] = c;
  }
  long long r2 = 1;
  out_ranks[0] = 1;
  for (int k = 1; k <= d; ++k) {
    long long c = r2 * n[k - 1];
    long long v = c < r1[k] ? c : r1[k];
    out_ranks[k] = (int32_t)v;
    r2 = v;
  }
  out_ranks[d] = 1;
  return T3F_OK;
}

extern "C" t3f_status t3f_device_status(const void* ws, t3f_stream_t stream) {
  if (!ws) return T3F_ERR_ARG;
  int32_t word = 0;
  if (cudaMemcpyAsync(&word, ws, sizeof(word), cudaMemcpyDeviceToHost,
                      (cudaStream_t)stream) != cudaSuccess)
    return T3F_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return T3F_ERR_CUDA;
  return (t3f_status)word;
}

extern "C" size_t t3f_workspace_size(int32_t op, const t3f_tt* a, const t3f_tt* b, int64_t n_items) {
  TTV va, vb;
  if (!a || make_view(a, &va, -1, a->m != nullptr) != T3F_OK) return 0;
  const bool need_b = op == T3F_OP_GRAM || op == T3F_OP_GRAM_BWD || op == T3F_OP_GRAM_BWD_TC ||
                      op == T3F_OP_RGATHER_BWD ||
                      op == T3F_OP_MATVEC || op == T3F_OP_MATVEC_BWD || op == T3F_OP_PSUM ||
                      op == T3F_OP_PSUM_BWD || op == T3F_OP_PROJECT || op == T3F_OP_TANGENT_GRAM ||
                      op == T3F_OP_COMPLETION_HVP;
  if (need_b && (!b || make_view(b, &vb, -1, b->m != nullptr) != T3F_OK)) return 0;
  switch (op) {
    case T3F_OP_GRAM: return kWsHeader;
    case T3F_OP_GRAM_BWD: return ws_gram_bwd(va, vb);
    case T3F_OP_GRAM_BWD_TC: return ws_gram_bwd_tc(va, vb);
    case T3F_OP_NORM: return ws_norm(va);
    case T3F_OP_GATHER: return ws_gather(va, n_items, false);
    case T3F_OP_GATHER_BWD: return ws_gather(va, n_items, true);
    case T3F_OP_RGATHER_BWD: return ws_rgather(va, vb, n_items);
    case T3F_OP_MATVEC: return kWsHeader;
    case T3F_OP_MATVEC_BWD: return 0;
    case T3F_OP_ORTH: return ws_orth(va);
    case T3F_OP_PSUM: return ws_psum(va, vb, false);
    case T3F_OP_PSUM_BWD: return ws_psum(va, vb, true);
    case T3F_OP_PROJECT: return ws_project(va, vb);
    case T3F_OP_TANGENT_GRAM: return ws_tangent_gram(va, vb);
    case T3F_OP_COMPLETION_HVP: return ws_completion_hvp(va, vb, n_items);
    case T3F_OP_ROUND: return ws_round(va);
    default: return 0;
  }
}

extern "C" int64_t t3f_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }
