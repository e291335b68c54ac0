// tune.cu -- plan autotuner and its on-disk cache.
//
// A plan's results do not depend on how its work is split (the passes are
// deterministic and chunk-invariant), only its speed does. The tuner times the
// candidate splits of a plan on synthetic inputs with CUDA events on the
// plan's stream and keeps the fastest:
//   uniform plans: the column solver (recursive filters or column FFTs, where
//                  both exist) x the pipeline split (one chunk of all fields,
//                  chunks sized for the L2 on two streams, halves, thirds and
//                  quarters of the batch, and for the recursive solve the
//                  largest chunks whose spectrum hand-off the plan keeps in L2
//                  on 2, 3 and 4 streams);
//   ragged plans:  the number of internal streams the per-item sub-plans are
//                  spread over.
// The winner is stored under a key naming the problem, the device and the
// library build, in a text cache (one "key<TAB>value" line per entry) that
// later plans read instead of timing again.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "gfc_build_id.h"
#include "gfc_internal.h"

using namespace gfc;

namespace {

std::mutex g_cache_mu;

__global__ void k_fill_pattern(float* x, long long n, unsigned seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    x[i] = ((float)(h & 0xffffu) / 65535.0f - 0.5f) * 0.02f;
  }
}

// device buffers for the timing runs: n elements of the plan's dtype each
struct TuneBufs {
  void* a = nullptr;
  void* b = nullptr;
  void* o = nullptr;
  ~TuneBufs() {
    cudaFree(a);
    cudaFree(b);
    cudaFree(o);
  }
};

cudaError_t make_bufs(TuneBufs& t, long long n, gfc_dtype dt, cudaStream_t st) {
  const size_t bytes = (size_t)n * dtype_size(dt);
  cudaError_t e = cudaMalloc(&t.a, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&t.b, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&t.o, bytes);
  // a pattern (as floats over the bytes: any bit pattern of 16-bit storage is
  // a finite small value or zero here, the solve's speed does not depend on it)
  if (e == cudaSuccess) {
    k_fill_pattern<<<1024, 256, 0, st>>>(static_cast<float*>(t.a), (long long)(bytes / 4), 17u);
    k_fill_pattern<<<1024, 256, 0, st>>>(static_cast<float*>(t.b), (long long)(bytes / 4), 29u);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// mean device time of `reps` solves on the plan's stream, after two untimed ones
gfc_status time_solve(gfc_plan* p, const TuneBufs& t, int reps, double* ms) {
  for (int i = 0; i < 2; ++i)
    if (gfc_status s = gfc_solve_from_gradient(p, t.a, t.b, t.o)) return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GFC_CUDA_TRY(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, p->stream);
  gfc_status st = GFC_OK;
  for (int i = 0; i < reps && e == cudaSuccess && st == GFC_OK; ++i) st = gfc_solve_from_gradient(p, t.a, t.b, t.o);
  if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float f = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != GFC_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "gfc_plan_autotune: timing");
  *ms = f / reps;
  return GFC_OK;
}

std::string device_tag(int dev) {
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "dev=?";
  char b[320];
  snprintf(b, sizeof b, "dev=%s sm=%d.%d sms=%d", pr.name, pr.major, pr.minor, pr.multiProcessorCount);
  for (char* c = b; *c; ++c)
    if (*c == '\t' || *c == '\n') *c = ' ';
  return b;
}

std::string plan_key(const gfc_plan* p) {
  char b[512];
  if (p->ragged) {
    // the items through their sub-plans and the generic fields
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](long long v) {
      h ^= (unsigned long long)v;
      h *= 1099511628211ull;
    };
    for (int j = 0; j < p->nsub; ++j) {
      const gfc_plan* q = p->sub[j];
      mix(q->H); mix(q->W); mix(q->C); mix(p->sub_off[j]);
    }
    mix(p->nfields);
    snprintf(b, sizeof b, "kind=ragged dtype=%d subplans=%d fields=%d items=%016llx", (int)p->dtype, p->nsub,
             p->nfields, h);
  } else {
    snprintf(b, sizeof b, "kind=uniform H=%d W=%d C=%d batch=%d dtype=%d pad=%d M=%d N=%d exact=%d", p->H, p->W,
             p->C, p->batch, (int)p->dtype, p->pad, p->M, p->N, p->exact ? 1 : 0);
  }
  return std::string("gfc-tune v1 build=") + GFC_BUILD_ID + " " + device_tag(p->device) + " " + b;
}

}  // namespace

extern "C" {

int gfc_tune_cache_get(const char* path, const char* key, char* value, int capacity) {
  clear_error();
  if (!path || !key || !value || capacity < 1) {
    fail(GFC_ERR_INVALID_ARG, "gfc_tune_cache_get: null argument");
    return -1;
  }
  std::lock_guard<std::mutex> lock(g_cache_mu);
  FILE* f = fopen(path, "r");
  if (!f) return 0;
  const size_t kl = strlen(key);
  std::vector<char> line(8192);
  int found = 0;
  while (fgets(line.data(), (int)line.size(), f)) {
    if (strncmp(line.data(), key, kl) == 0 && line[kl] == '\t') {
      char* v = line.data() + kl + 1;
      v[strcspn(v, "\r\n")] = 0;
      snprintf(value, (size_t)capacity, "%s", v);
      found = 1;  // the last entry for a key wins
    }
  }
  fclose(f);
  return found;
}

gfc_status gfc_tune_cache_put(const char* path, const char* key, const char* value) {
  clear_error();
  if (!path || !key || !value) return fail(GFC_ERR_INVALID_ARG, "gfc_tune_cache_put: null argument");
  if (strpbrk(key, "\t\n") || strpbrk(value, "\t\n"))
    return fail(GFC_ERR_INVALID_ARG, "gfc_tune_cache_put: key and value may not hold tabs or newlines");
  std::lock_guard<std::mutex> lock(g_cache_mu);
  std::string keep;
  const size_t kl = strlen(key);
  if (FILE* f = fopen(path, "r")) {  // every other entry is kept
    std::vector<char> line(8192);
    while (fgets(line.data(), (int)line.size(), f))
      if (!(strncmp(line.data(), key, kl) == 0 && line[kl] == '\t')) keep += line.data();
    fclose(f);
  }
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return fail(GFC_ERR_INVALID_ARG, "gfc_tune_cache_put: cannot write %s", tmp.c_str());
  const bool ok = fputs(keep.c_str(), f) >= 0 && fprintf(f, "%s\t%s\n", key, value) > 0;
  if (fclose(f) != 0 || !ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return fail(GFC_ERR_INVALID_ARG, "gfc_tune_cache_put: cannot write %s", path);
  }
  return GFC_OK;
}

gfc_status gfc_plan_tune_key(const gfc_plan* plan, char* key, int capacity) {
  clear_error();
  if (!plan || !key || capacity < 1) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_tune_key: null argument");
  const std::string k = plan_key(plan);
  if ((int)k.size() >= capacity) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_tune_key: buffer too small");
  memcpy(key, k.c_str(), k.size() + 1);
  return GFC_OK;
}

gfc_status gfc_plan_autotune(gfc_plan* plan, const char* cache_path, gfc_tune_result* out) {
  clear_error();
  if (!plan) return fail(GFC_ERR_INVALID_ARG, "gfc_plan_autotune: null plan");
  if (plan->profiling) return fail(GFC_ERR_UNSUPPORTED, "gfc_plan_autotune: turn profiling off first");
  gfc_tune_result r;
  memset(&r, 0, sizeof r);
  const std::string key = plan_key(plan);
  char cached[256] = {0};
  const bool hit = cache_path && gfc_tune_cache_get(cache_path, key.c_str(), cached, sizeof cached) == 1;
  clear_error();
  GFC_CUDA_TRY(cudaStreamSynchronize(plan->stream));

  if (plan->ragged) {
    int best = plan->rag_active, n = 0;
    double best_ms = 0.0;
    if (plan->nsub > 1) {
      if (hit && sscanf(cached, "rag_streams=%d", &best) == 1) {
        r.from_cache = 1;
      } else {
        long long total = 0;
        for (int j = 0; j < plan->nsub; ++j) {
          const gfc_plan* q = plan->sub[j];
          total = std::max(total, plan->sub_off[j] + (long long)q->C * q->H * q->W);
        }
        total = std::max(total, plan->rag_total);
        TuneBufs t;
        GFC_CUDA_TRY(make_bufs(t, total, plan->dtype, plan->stream));
        for (int k : {1, 2, 4, 8}) {
          if (k > plan->nsub && k > 1) break;
          if (gfc_status s = ragged_set_streams(plan, k)) return s;
          double ms = 0.0;
          if (gfc_status s = time_solve(plan, t, 3, &ms)) return s;
          ++n;
          if (best_ms == 0.0 || ms < best_ms) {
            best_ms = ms;
            best = k;
          }
        }
      }
      if (gfc_status s = ragged_set_streams(plan, best)) return s;
    }
    r.rag_streams = plan->rag_active;
    r.ms = best_ms;
    r.candidates = n;
    if (cache_path && !r.from_cache && n > 0) {
      char v[64];
      snprintf(v, sizeof v, "rag_streams=%d", r.rag_streams);
      if (gfc_status s = gfc_tune_cache_put(cache_path, key.c_str(), v)) return s;
    }
    if (out) *out = r;
    return GFC_OK;
  }

  // uniform plans: candidate options
  gfc_plan_opts base;
  memset(&base, 0, sizeof base);
  base.H = plan->H; base.W = plan->W; base.C = plan->C; base.batch = plan->batch; base.dtype = plan->dtype;
  base.pad = plan->pad; base.size_policy = plan->exact ? GFC_SIZE_EXACT : GFC_SIZE_SMOOTH;
  base.stream = plan->stream; base.streams = 1;
  base.column_solver = plan->tri ? GFC_COLUMN_RECURSIVE : GFC_COLUMN_FFT;
  base.block_items = 0;
  gfc_plan_opts cand[24];  // (a plain array: the options type is an unnamed struct)
  int ncand = 0;
  const long fields = (long)plan->batch * plan->C;
  // scratch the passes hand off per field (the packed rows only when pass L runs)
  const size_t per_field = ((size_t)plan->spec_field + plan->tri_field) * sizeof(float2);
  const int nsolvers = plan->fast_cols ? 2 : 1;
  for (int si = 0; si < nsolvers; ++si) {
    gfc_plan_opts o = base;
    o.column_solver = si == 0 ? GFC_COLUMN_RECURSIVE : GFC_COLUMN_FFT;
    cand[ncand++] = o;  // one chunk
    // chunks whose scratch fits 32 or 64 MB of L2, and halves and quarters of
    // the batch, two streams (one chunk's carry sweep and inverse pass can
    // overlap the next chunk's row pass)
    const long cs[6] = {(long)(((size_t)32 << 20) / (per_field ? per_field : 1)),
                        (long)(((size_t)64 << 20) / (per_field ? per_field : 1)), (fields + 1) / 2, (fields + 3) / 4,
                        (fields + 2) / 3, (fields + 3) / 4};
    const int ss[6] = {2, 2, 2, 2, 3, 4};  // streams of each split
    for (int i = 0; i < 6 && ncand < 22; ++i) {
      const long c = cs[i];
      bool dup = false;
      for (int j = 0; j < i; ++j) dup = dup || (cs[j] == c && ss[j] == ss[i]);
      if (c >= 1 && c < fields && !dup) {
        o.chunk = (int)c;
        o.streams = ss[i];
        cand[ncand++] = o;
        if (si == 0 && plan->fast) {  // the same split with one block per item
          o.block_items = 1;
          cand[ncand++] = o;
          o.block_items = 0;
        }
        o.chunk = 0;
        o.streams = 1;
      }
    }
    // recursive column solve: the largest chunks whose spectrum hand-off fits
    // the L2 budget on 2, 3 and 4 streams (the plan then keeps it in L2)
    for (int ns = 2; si == 0 && plan->tri && ns <= 4 && ncand < 22; ++ns) {
      const long c = (long)(kL2ResidentBytes / ((size_t)ns * tri_handoff_bytes(plan)));
      bool dup = false;
      for (int j = 0; j < ncand; ++j) dup = dup || (cand[j].chunk == c && cand[j].streams == ns);
      if (c >= 1 && c < fields && !dup) {
        o.chunk = (int)c;
        o.streams = ns;
        cand[ncand++] = o;
        o.chunk = 0;
        o.streams = 1;
      }
    }
    if (si == 0 && plan->fast && ncand < 24) {  // one chunk, one block per item
      o.block_items = 1;
      cand[ncand++] = o;
      o.block_items = 0;
    }
  }
  gfc_plan_opts best = base;
  double best_ms = 0.0;
  int n = 0;
  if (hit && sscanf(cached, "column_solver=%d chunk=%d streams=%d block_items=%d", &best.column_solver, &best.chunk,
                    &best.streams, &best.block_items) == 4) {
    r.from_cache = 1;
  } else {
    TuneBufs t;
    GFC_CUDA_TRY(make_bufs(t, fields * (long long)plan->H * plan->W, plan->dtype, plan->stream));
    for (int ci = 0; ci < ncand; ++ci) {
      const gfc_plan_opts& o = cand[ci];
      gfc_plan* q = nullptr;
      if (gfc_status s = gfc_plan_create_ex(&q, &o)) return s;
      double ms = 0.0;
      gfc_status s = time_solve(q, t, 5, &ms);
      gfc_destroy(q);
      if (s != GFC_OK) return s;
      ++n;
      if (best_ms == 0.0 || ms < best_ms) {
        best_ms = ms;
        best = o;
      }
    }
  }
  // the winner replaces the plan's contents; the handle stays the caller's
  gfc_plan* w = nullptr;
  if (gfc_status s = gfc_plan_create_ex(&w, &best)) return s;
  w->profiling = false;
  gfc_plan tmp = *plan;
  *plan = *w;
  *w = tmp;
  gfc_destroy(w);
  r.column_solver = best.column_solver;
  r.block_items = best.block_items;
  r.chunk = plan->chunk;
  r.streams = plan->nslots;
  r.l2_resident = plan->l2res ? 1 : 0;
  r.ms = best_ms;
  r.candidates = n;
  if (cache_path && !r.from_cache && n > 0) {
    char v[96];
    snprintf(v, sizeof v, "column_solver=%d chunk=%d streams=%d block_items=%d", best.column_solver, best.chunk,
             best.streams, best.block_items);
    if (gfc_status s = gfc_tune_cache_put(cache_path, key.c_str(), v)) return s;
  }
  if (out) *out = r;
  return GFC_OK;
}

}  // extern "C"
