// Launch-geometry autotuner and its cache.
//
// The paper's only tuning knob is the compile-time maximum rank (Algorithm 8); on the GPU
// the launch geometry matters as much: threads per CTA, elements per tile and resident
// CTAs per SM.  triot_autotune times candidates with CUDA events on the caller's buffers
// and caches the fastest per (GPU, op, dtype, effective rank, inner-extent class).  The
// cache persists as JSON.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/triot.h"
#include "internal.h"

namespace triot {

namespace {

std::mutex g_mu;
std::map<std::string, TuneCfg> g_cache;

int inner_class(long long inner) {
  int c = 0;
  while (c < 40 && (1ll << (c + 1)) <= inner) ++c;
  return c;  // floor(log2(inner))
}

std::string make_key(int op, int dtype, const Canon& c) {
  DeviceInfo dev;
  const char* name = "gpu";
  if (device_info(dev) == TRIOT_OK) name = dev.name;
  char buf[256];
  snprintf(buf, sizeof buf, "%s|op%d|dt%d|D%d|in%d", name, op, dtype, c.D,
           inner_class(c.ext[c.D > 0 ? c.D - 1 : 0]));
  return buf;
}

int canon_for(int op, int rank, const int64_t* xshape, const int64_t* yshape, Canon& c) {
  std::string err;
  int st;
  if (op == TRIOT_OP_MOMENT) {
    st = canon_moment(rank, xshape, c, err);
  } else {
    const int rop = op == TRIOT_OP_EMBED ? ROW_EMBED : op == TRIOT_OP_CROP ? ROW_CROP : ROW_PRODUCT;
    bool xe = false;
    st = canon_rows(rop, rank, xshape, yshape, c, xe, err);
  }
  if (st) return fail(st, err);
  return TRIOT_OK;
}

bool valid_tune(const triot_tune& t) {
  if (t.threads && (t.threads < 32 || t.threads > 1024 || t.threads % 32)) return false;
  if (t.tile_elems < 0 || t.ctas_per_sm < 0 || t.ctas_per_sm > 32 || t.unroll < 0 || t.unroll > 8) return false;
  return true;
}

}  // namespace

TuneCfg tune_lookup(int op, int dtype, const Canon& c) {
  const std::string k = make_key(op, dtype, c);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(k);
  return it == g_cache.end() ? TuneCfg() : it->second;
}

void tune_store(int op, int dtype, const Canon& c, const TuneCfg& t) {
  const std::string k = make_key(op, dtype, c);
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[k] = t;
}

// A batch is keyed by its dtype, mode and size class: floor(log2) of its pair count and of
// its total number of y elements.
std::string batch_key(int dtype, int mode, long long npairs, long long ny_total) {
  DeviceInfo dev;
  const char* name = "gpu";
  if (device_info(dev) == TRIOT_OK) name = dev.name;
  char buf[256];
  snprintf(buf, sizeof buf, "%s|op%d|dt%d|mode%d|n%d|y%d", name, TRIOT_OP_BATCH, dtype, mode,
           inner_class(npairs), inner_class(ny_total));
  return buf;
}

TuneCfg tune_lookup_key(const std::string& k) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(k);
  return it == g_cache.end() ? TuneCfg() : it->second;
}

void tune_store_key(const std::string& k, const TuneCfg& t) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[k] = t;
}

}  // namespace triot

using namespace triot;

extern "C" {

int triot_tune_get(int op, int rank, const int64_t* xshape, const int64_t* yshape, int dtype,
                   triot_tune* out) {
  if (!out) return fail(TRIOT_ERR_NULL, "out is NULL");
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  Canon c;
  int st = canon_for(op, rank, xshape, yshape, c);
  if (st) return st;
  const TuneCfg t = tune_lookup(op, dtype, c);
  out->threads = t.threads;
  out->tile_elems = t.tile_elems;
  out->ctas_per_sm = t.ctas_per_sm;
  out->unroll = t.unroll;
  return ok();
}

int triot_tune_set(int op, int rank, const int64_t* xshape, const int64_t* yshape, int dtype,
                   const triot_tune* tune) {
  if (!tune) return fail(TRIOT_ERR_NULL, "tune is NULL");
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  if (!valid_tune(*tune)) return fail(TRIOT_ERR_ARG, "tuning values out of range");
  Canon c;
  int st = canon_for(op, rank, xshape, yshape, c);
  if (st) return st;
  TuneCfg t;
  t.threads = tune->threads;
  t.tile_elems = tune->tile_elems;
  t.ctas_per_sm = tune->ctas_per_sm;
  t.unroll = tune->unroll;
  tune_store(op, dtype, c, t);
  return ok();
}

int triot_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
  return ok();
}

int triot_tune_save(const char* path) {
  if (!path) return fail(TRIOT_ERR_NULL, "path is NULL");
  FILE* f = fopen(path, "w");
  if (!f) return fail(TRIOT_ERR_ARG, std::string("cannot open ") + path);
  std::lock_guard<std::mutex> lk(g_mu);
  fprintf(f, "{\"triot_tune\": 1, \"entries\": [\n");
  size_t i = 0;
  for (const auto& kv : g_cache) {
    fprintf(f, "  {\"key\": \"%s\", \"threads\": %d, \"tile_elems\": %d, \"ctas_per_sm\": %d, \"unroll\": %d}%s\n",
            kv.first.c_str(), kv.second.threads, kv.second.tile_elems, kv.second.ctas_per_sm,
            kv.second.unroll, (++i < g_cache.size()) ? "," : "");
  }
  fprintf(f, "]}\n");
  fclose(f);
  return ok();
}

int triot_tune_load(const char* path) {
  if (!path) return fail(TRIOT_ERR_NULL, "path is NULL");
  FILE* f = fopen(path, "r");
  if (!f) return fail(TRIOT_ERR_ARG, std::string("cannot open ") + path);
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
  fclose(f);
  // one entry per object: {"key": "...", "threads": N, "tile_elems": N, "ctas_per_sm": N, "unroll": N}
  size_t pos = 0;
  int loaded = 0;
  std::map<std::string, TuneCfg> add;
  while ((pos = text.find("\"key\"", pos)) != std::string::npos) {
    const size_t q1 = text.find('"', text.find(':', pos) + 1);
    const size_t q2 = text.find('"', q1 + 1);
    if (q1 == std::string::npos || q2 == std::string::npos) break;
    const std::string key = text.substr(q1 + 1, q2 - q1 - 1);
    const size_t end = text.find('}', q2);
    const std::string obj = text.substr(q2, end - q2);
    TuneCfg t;
    auto field = [&](const char* name, int& v) {
      const size_t p = obj.find(name);
      if (p != std::string::npos) v = atoi(obj.c_str() + obj.find(':', p) + 1);
    };
    field("\"threads\"", t.threads);
    field("\"tile_elems\"", t.tile_elems);
    field("\"ctas_per_sm\"", t.ctas_per_sm);
    field("\"unroll\"", t.unroll);
    triot_tune tt{t.threads, t.tile_elems, t.ctas_per_sm, t.unroll};
    if (!valid_tune(tt)) return fail(TRIOT_ERR_ARG, "tuning file holds out-of-range values");
    add[key] = t;
    ++loaded;
    pos = end == std::string::npos ? text.size() : end;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  for (const auto& kv : add) g_cache[kv.first] = kv.second;
  return ok();
}

int triot_autotune(int op, int rank, const int64_t* xshape, const void* x, const int64_t* yshape,
                   void* y, int dtype, void* workspace, size_t workspace_bytes, void* stream,
                   triot_tune* best) {
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  if (op < TRIOT_OP_EMBED || op > TRIOT_OP_MOMENT) return fail(TRIOT_ERR_ARG, "op cannot be autotuned here");
  Canon c;
  int st = canon_for(op, rank, xshape, yshape, c);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int es = dtype_size(dtype);
  std::vector<TuneCfg> cands;
  if (op == TRIOT_OP_MOMENT) {
    for (int cps : {1, 2, 3, 4, 6, 8}) {
      TuneCfg t;
      t.ctas_per_sm = cps;
      cands.push_back(t);
    }
  } else {
    const int base = 32768 / es;
    for (int th : {128, 256, 512})
      for (int tile : {base / 4, base / 2, base, base * 2})
        for (int cps : {2, 4, 8}) {
          TuneCfg t;
          t.threads = th;
          t.tile_elems = tile;
          t.ctas_per_sm = cps;
          cands.push_back(t);
        }
  }
  double* out = nullptr;
  cudaError_t e;
  if (op == TRIOT_OP_MOMENT) {
    e = cudaMallocAsync((void**)&out, sizeof(double) * (rank + 1), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
  }
  auto run = [&](const TuneCfg& t) -> int {
    if (op == TRIOT_OP_MOMENT) return moment_call(rank, xshape, x, dtype, out, workspace, workspace_bytes, s, &t);
    const int rop = op == TRIOT_OP_EMBED ? ROW_EMBED : op == TRIOT_OP_CROP ? ROW_CROP : ROW_PRODUCT;
    // same argument order as triot_embed / triot_crop / triot_product (crop writes x)
    return launch_rows(rop, rank, xshape, x, yshape, y, dtype, 0, s, &t);
  };
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best_ms = 1e30f;
  TuneCfg best_t;
  int rc = TRIOT_OK;
  for (const TuneCfg& t : cands) {
    if ((rc = run(t))) break;  // warm-up (also validates the candidate)
    std::vector<float> ms;
    for (int r = 0; r < 5 && rc == TRIOT_OK; ++r) {
      cudaEventRecord(a, s);
      rc = run(t);
      cudaEventRecord(b, s);
      cudaEventSynchronize(b);
      float v = 0.f;
      cudaEventElapsedTime(&v, a, b);
      ms.push_back(v);
    }
    if (rc) break;
    std::sort(ms.begin(), ms.end());
    if (ms[ms.size() / 2] < best_ms) { best_ms = ms[ms.size() / 2]; best_t = t; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (out) cudaFreeAsync(out, s);
  e = cudaStreamSynchronize(s);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  tune_store(op, dtype, c, best_t);
  if (best) {
    best->threads = best_t.threads;
    best->tile_elems = best_t.tile_elems;
    best->ctas_per_sm = best_t.ctas_per_sm;
    best->unroll = best_t.unroll;
  }
  return ok();
}

}  // extern "C"
