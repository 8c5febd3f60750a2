// Autotuner of the sampler's launch configuration and its table.
//
// The blocked sampler of Algorithm 4 has a few free choices that decide its
// speed on a given GPU, and the paper tunes its analogues (tile and block
// sizes) by hand per machine (Section 4). Here they are measured:
//   - outer block width (columns contracted per tensor-core update),
//   - panel pipeline of the mixed real paths (single helper, chunked, or
//     split: the decisions on a few CTAs, the rows below in a wide launch),
//   - draws in flight, and with them the per-launch CTA cap (SMs / streams):
//     one draw leaves most SMs idle during its sequential decisions, so
//     several draws on several streams fill them.
// dpp_autotune times every candidate on the caller's kernel and keeps the
// fastest in a table keyed by (GPU name, SM count, op, dtype, precision,
// floor(log2 n)); every later call with that key runs with the entry's
// configuration (begin_call). The table is saved and loaded as JSON, and the
// file named by DPP_TUNE_CACHE is loaded with the library.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "dpp.h"
#include "dpp_internal.h"

namespace dpp {
namespace {

struct Entry {
  std::string gpu;
  int sms = 0;
  dpp_tune_entry e{};
};

std::mutex g_mu;
std::vector<Entry> g_table;

// Configuration forced by dpp_autotune on the thread that runs a candidate.
thread_local const dpp_tune_entry* tl_force = nullptr;

int bucket_of(int64_t n) {
  int b = 0;
  while (n > 1) {
    n >>= 1;
    ++b;
  }
  return b;
}

struct GpuId {
  std::string name;
  int sms = 0;
  bool ok = false;
};

// Name and SM count of the current device (cached per device).
bool gpu_id(GpuId* out) {
  static GpuId cache[64];
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lk(mu);
  if (!cache[dev].ok) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return false;
    cache[dev].name = p.name;
    cache[dev].sms = p.multiProcessorCount;
    cache[dev].ok = true;
  }
  *out = cache[dev];
  return true;
}

bool same_key(const Entry& a, const std::string& gpu, int sms, const dpp_tune_entry& e) {
  return a.gpu == gpu && a.sms == sms && a.e.op == e.op && a.e.dtype == e.dtype &&
         a.e.precision == e.precision && a.e.n_bucket == e.n_bucket;
}

void put(const std::string& gpu, int sms, const dpp_tune_entry& e) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (Entry& x : g_table) {
    if (same_key(x, gpu, sms, e)) {
      x.e = e;
      return;
    }
  }
  Entry x;
  x.gpu = gpu;
  x.sms = sms;
  x.e = e;
  g_table.push_back(x);
}

bool find(int32_t op, int64_t n, int32_t dtype, int32_t precision, dpp_tune_entry* out) {
  GpuId id;
  if (!gpu_id(&id)) return false;
  dpp_tune_entry k{};
  k.op = op;
  k.dtype = dtype;
  k.precision = precision;
  k.n_bucket = bucket_of(n);
  std::lock_guard<std::mutex> lk(g_mu);
  for (const Entry& x : g_table) {
    if (same_key(x, id.name, id.sms, k)) {
      *out = x.e;
      return true;
    }
  }
  return false;
}

void apply(const dpp_tune_entry& e, Tuning* t) {
  if (e.op == kOpBatched) {
    t->batched_threads = e.batched_threads;
    return;
  }
  if (e.outer_block >= 32) t->outer_block = e.outer_block;
  t->panel_pipeline = e.panel_pipeline;
  t->max_ctas = e.max_ctas;
  t->update_variant = e.update_variant;
}

// ---------------------------------------------------------------------------
// JSON: {"version": 1, "entries": [{"gpu": "...", "sms": 152, "op": 0, ...}]}
// A flat reader for exactly this shape: objects of string and number fields.
// ---------------------------------------------------------------------------
const char* skip_ws(const char* p) {
  while (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t' || *p == ',') ++p;
  return p;
}

bool read_string(const char** pp, std::string* out) {
  const char* p = *pp;
  if (*p != '"') return false;
  ++p;
  out->clear();
  while (*p && *p != '"') {
    if (*p == '\\' && p[1]) ++p;
    out->push_back(*p++);
  }
  if (*p != '"') return false;
  *pp = p + 1;
  return true;
}

// Parse one flat object starting at '{'; fills an entry. Returns false on a
// syntax error.
bool read_entry(const char** pp, Entry* x) {
  const char* p = skip_ws(*pp);
  if (*p != '{') return false;
  ++p;
  while (true) {
    p = skip_ws(p);
    if (*p == '}') {
      *pp = p + 1;
      return true;
    }
    std::string key;
    if (!read_string(&p, &key)) return false;
    p = skip_ws(p);
    if (*p != ':') return false;
    p = skip_ws(p + 1);
    if (*p == '"') {
      std::string v;
      if (!read_string(&p, &v)) return false;
      if (key == "gpu") x->gpu = v;
    } else {
      char* end = nullptr;
      const double v = strtod(p, &end);
      if (end == p) return false;
      p = end;
      dpp_tune_entry& e = x->e;
      if (key == "sms") x->sms = (int)v;
      else if (key == "op") e.op = (int32_t)v;
      else if (key == "dtype") e.dtype = (int32_t)v;
      else if (key == "precision") e.precision = (int32_t)v;
      else if (key == "n_bucket") e.n_bucket = (int32_t)v;
      else if (key == "n") e.n = (int64_t)v;
      else if (key == "outer_block") e.outer_block = (int32_t)v;
      else if (key == "panel_pipeline") e.panel_pipeline = (int32_t)v;
      else if (key == "max_ctas") e.max_ctas = (int32_t)v;
      else if (key == "streams") e.streams = (int32_t)v;
      else if (key == "samples_per_s") e.samples_per_s = v;
      else if (key == "candidates") e.candidates = (int32_t)v;
      else if (key == "update_variant") e.update_variant = (int32_t)v;
      else if (key == "batched_threads") e.batched_threads = (int32_t)v;
    }
  }
}

bool valid(const Entry& x) {
  const dpp_tune_entry& e = x.e;
  if (e.op == kOpBatched)
    return !x.gpu.empty() && x.sms > 0 && e.dtype == DPP_R64 && e.precision == DPP_PREC_FP32 &&
           e.n_bucket >= 0 && e.n_bucket < 40 && (e.batched_threads == 128 || e.batched_threads == 256);
  return !x.gpu.empty() && x.sms > 0 && e.batched_threads == 0 && e.op >= 0 && e.op <= 1 &&
         (e.dtype == 0 || e.dtype == 1) &&
         e.precision >= 0 && e.precision <= 2 && e.n_bucket >= 0 && e.n_bucket < 40 &&
         (e.outer_block == 0 || (e.outer_block >= 32 && e.outer_block <= kMaxOuterBlock &&
                                 e.outer_block % 32 == 0)) &&
         e.panel_pipeline >= 0 && e.panel_pipeline <= 3 && e.max_ctas >= 0 &&
         e.max_ctas <= 4096 && e.streams >= 1 && e.streams <= 64 && e.update_variant >= 0 &&
         e.update_variant <= 3;
}

int load_file(const char* path, std::string* err) {
  FILE* f = fopen(path, "rb");
  if (!f) {
    *err = std::string("cannot open ") + path;
    return -1;
  }
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
  fclose(f);
  const char* p = strstr(text.c_str(), "\"entries\"");
  if (!p) {
    *err = "no \"entries\" array";
    return -1;
  }
  p = strchr(p, '[');
  if (!p) {
    *err = "no \"entries\" array";
    return -1;
  }
  ++p;
  std::vector<Entry> got;
  while (true) {
    p = skip_ws(p);
    if (*p == ']') break;
    Entry x;
    if (!read_entry(&p, &x)) {
      *err = "malformed entry";
      return -1;
    }
    if (!valid(x)) {
      *err = "entry out of range";
      return -1;
    }
    got.push_back(x);
  }
  for (const Entry& x : got) put(x.gpu, x.sms, x.e);
  return (int)got.size();
}

struct EnvLoad {
  EnvLoad() {
    const char* path = getenv("DPP_TUNE_CACHE");
    if (path && *path) {
      std::string err;
      if (load_file(path, &err) < 0) fprintf(stderr, "dpp: DPP_TUNE_CACHE: %s\n", err.c_str());
    }
  }
} g_env_load;

// ---------------------------------------------------------------------------
// Timing of candidates
// ---------------------------------------------------------------------------
struct Scratch {
  char* ws;
  uint8_t* keep;
  dpp_result* res;
};

dpp_status run_candidate(int32_t op, const void* K, int64_t n, int64_t ld, int32_t dtype,
                         int32_t precision, const dpp_tune_entry& c, int draws,
                         const std::vector<Scratch>& scr, size_t need,
                         const std::vector<cudaStream_t>& st, cudaStream_t caller,
                         cudaEvent_t e0, cudaEvent_t e1, const std::vector<cudaEvent_t>& done,
                         double* sps) {
  tl_force = &c;
  auto draw = [&](int s, uint64_t seed) -> dpp_status {
    const Scratch& x = scr[s];
    return op == DPP_OP_SAMPLE_HERMITIAN
               ? dpp_sample_hermitian(K, n, ld, dtype, precision, seed, 0, nullptr, x.keep,
                                      nullptr, nullptr, x.res, x.ws, need, st[s])
               : dpp_sample_lu(K, n, ld, dtype, precision, seed, 0, nullptr, x.keep, nullptr,
                               nullptr, x.res, x.ws, need, st[s]);
  };
  dpp_status rs = DPP_OK;
  const int S = c.streams;
  cudaError_t e = cudaEventRecord(e0, caller);
  for (int s = 0; s < S && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(st[s], e0, 0);
  for (int s = 0; s < S && rs == DPP_OK && e == cudaSuccess; ++s) rs = draw(s, 1000000u + s);
  if (rs == DPP_OK && e == cudaSuccess) {
    for (int s = 0; s < S && e == cudaSuccess; ++s) e = cudaEventRecord(done[s], st[s]);
    for (int s = 0; s < S && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(caller, done[s], 0);
    if (e == cudaSuccess) e = cudaEventRecord(e0, caller);
    for (int s = 0; s < S && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(st[s], e0, 0);
    for (int d = 0; d < draws && rs == DPP_OK && e == cudaSuccess; ++d) rs = draw(d % S, d);
    for (int s = 0; s < S && e == cudaSuccess; ++s) e = cudaEventRecord(done[s], st[s]);
    for (int s = 0; s < S && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(caller, done[s], 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, caller);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  }
  tl_force = nullptr;
  if (rs != DPP_OK) return rs;
  if (e != cudaSuccess) return set_last_cuda_error(e, "dpp_autotune");
  float ms = 0.f;
  e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess) return set_last_cuda_error(e, "dpp_autotune: timing");
  *sps = ms > 0.f ? draws / (ms * 1e-3) : 0.0;
  return DPP_OK;
}

size_t per_stream_bytes(int32_t op, int64_t n, int32_t dtype, int32_t precision) {
  const size_t need = dpp_workspace_size(op, n, dtype, precision, op == DPP_OP_SAMPLE_HERMITIAN);
  if (!need) return 0;
  return align256(need) + align256((size_t)(n > 0 ? n : 1)) + 256;
}

}  // namespace

void begin_call(int32_t op, int64_t n, int32_t dtype, int32_t precision) {
  g_tuning = g_settings;
  if (tl_force) {
    apply(*tl_force, &g_tuning);
    return;
  }
  if (!g_settings.use_cache) return;
  dpp_tune_entry e;
  if (find(op, n, dtype, precision, &e)) apply(e, &g_tuning);
}

}  // namespace dpp

using namespace dpp;

extern "C" {

size_t dpp_autotune_workspace_size(int32_t op, int64_t n, int32_t dtype, int32_t precision,
                                   int32_t max_streams) {
  if ((op != DPP_OP_SAMPLE_HERMITIAN && op != DPP_OP_SAMPLE_LU) || n < 1 || max_streams < 1 ||
      max_streams > 8)
    return 0;
  const size_t per = per_stream_bytes(op, n, dtype, precision);
  return per ? (size_t)max_streams * per + 256 : 0;
}

dpp_status dpp_autotune(int32_t op, const void* K, int64_t n, int64_t ld, int32_t dtype,
                        int32_t precision, int32_t max_streams, int32_t draws, void* workspace,
                        size_t workspace_bytes, dpp_tune_entry* best, void* stream) {
  clear_last_error();
  if (op != DPP_OP_SAMPLE_HERMITIAN && op != DPP_OP_SAMPLE_LU)
    return set_last_error(DPP_ERR_INVALID_ARG, "dpp_autotune: op must be a sampler");
  if (n < 1 || ld < n || !K) return set_last_error(DPP_ERR_INVALID_ARG, "dpp_autotune: bad K / n / ld");
  if (max_streams < 1 || max_streams > 8)
    return set_last_error(DPP_ERR_INVALID_ARG, "dpp_autotune: max_streams must be in [1, 8]");
  if (draws < 1 || draws > 4096)
    return set_last_error(DPP_ERR_INVALID_ARG, "dpp_autotune: draws must be in [1, 4096]");
  const size_t need = dpp_workspace_size(op, n, dtype, precision, op == DPP_OP_SAMPLE_HERMITIAN);
  if (!need) return set_last_error(DPP_ERR_UNSUPPORTED, "dpp_autotune: unsupported combination");
  const size_t per = per_stream_bytes(op, n, dtype, precision);
  if (!workspace || ((uintptr_t)workspace & 255))
    return set_last_error(DPP_ERR_WORKSPACE, "dpp_autotune: workspace must be 256-byte aligned");
  if (workspace_bytes < (size_t)max_streams * per + 256)
    return set_last_error(DPP_ERR_WORKSPACE, "dpp_autotune: workspace too small");
  GpuId id;
  if (!gpu_id(&id)) return set_last_error(DPP_ERR_CUDA, "dpp_autotune: no current device");

  // candidates
  const bool mixed = precision != DPP_PREC_FP64;
  std::vector<dpp_tune_entry> cand;
  const int stream_opts[4] = {1, 2, 4, 8};
  for (int so : stream_opts) {
    if (so > max_streams) continue;
    const int cap = so == 1 ? 0 : (id.sms / so < 8 ? 8 : id.sms / so);
    const int nouter = mixed ? 2 : 1;
    for (int oi = 0; oi < nouter; ++oi) {
      // (the complex LU path takes outer blocks of at most 128 columns)
      const bool cxlu = op == DPP_OP_SAMPLE_LU && dtype == DPP_C128;
      const int outer = mixed ? (oi == 0 ? (cxlu ? 128 : 256) : (cxlu ? 64 : 128)) : 0;
      // panel pipelines: single helper, chunked and split for real Hermitian
      // draws; chunked (0) and split for real LU draws; none to choose else
      int pipes[3] = {0, 0, 0}, npipe = 1;
      if (mixed && dtype == DPP_R64 && op == DPP_OP_SAMPLE_HERMITIAN) {
        pipes[0] = 1, pipes[1] = 2, pipes[2] = 3, npipe = 3;
      } else if (mixed && dtype == DPP_R64) {
        pipes[0] = 0, pipes[1] = 3, npipe = 2;
      }
      for (int pi = 0; pi < npipe; ++pi) {
        const int pipe = pipes[pi];
        dpp_tune_entry c{};
        c.op = op;
        c.dtype = dtype;
        c.precision = precision;
        c.n = n;
        c.n_bucket = bucket_of(n);
        c.outer_block = outer;
        c.panel_pipeline = pipe;
        c.max_ctas = cap;
        c.streams = so;
        cand.push_back(c);
      }
    }
  }

  std::vector<Scratch> scr((size_t)max_streams);
  char* base = static_cast<char*>(workspace);
  for (int s = 0; s < max_streams; ++s) {
    char* p = base + (size_t)s * per;
    scr[s].ws = p;
    scr[s].keep = reinterpret_cast<uint8_t*>(p + align256(need));
    scr[s].res = reinterpret_cast<dpp_result*>(p + align256(need) + align256((size_t)n));
  }
  std::vector<cudaStream_t> st((size_t)max_streams, nullptr);
  std::vector<cudaEvent_t> done((size_t)max_streams, nullptr);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int s = 0; s < max_streams && e == cudaSuccess; ++s) {
    e = cudaStreamCreateWithFlags(&st[s], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[s], cudaEventDisableTiming);
  }
  dpp_status rs = e == cudaSuccess ? DPP_OK : set_last_cuda_error(e, "dpp_autotune: set-up");
  dpp_tune_entry win{};
  double win_sps = -1.0;
  for (size_t i = 0; i < cand.size() && rs == DPP_OK; ++i) {
    double sps = 0.0;
    rs = run_candidate(op, K, n, ld, dtype, precision, cand[i], draws, scr, need, st,
                       static_cast<cudaStream_t>(stream), e0, e1, done, &sps);
    if (rs == DPP_OK && sps > win_sps) {
      win_sps = sps;
      win = cand[i];
      win.samples_per_s = sps;
    }
  }
  // second pass: the tensor-core update variants with the winner's settings
  int ncand = (int)cand.size();
  if (rs == DPP_OK && mixed) {
    const int nv = precision == DPP_PREC_3XTF32 ? 3 : 1;
    for (int v = 1; v <= nv && rs == DPP_OK; ++v) {
      dpp_tune_entry c = win;
      c.update_variant = v;
      double sps = 0.0;
      rs = run_candidate(op, K, n, ld, dtype, precision, c, draws, scr, need, st,
                         static_cast<cudaStream_t>(stream), e0, e1, done, &sps);
      ++ncand;
      if (rs == DPP_OK && sps > win_sps) {
        win_sps = sps;
        win = c;
        win.samples_per_s = sps;
      }
    }
  }
  cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  for (int s = 0; s < max_streams; ++s) {
    if (st[s]) cudaStreamDestroy(st[s]);
    if (done[s]) cudaEventDestroy(done[s]);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rs != DPP_OK) return rs;
  win.candidates = (int32_t)ncand;
  put(id.name, id.sms, win);
  if (best) *best = win;
  return DPP_OK;
}

dpp_status dpp_autotune_batched(int32_t batch, const int64_t* n, const double* const* K,
                                const int64_t* ld, int64_t n_max, uint64_t seed,
                                uint8_t* const* keep, dpp_result* results, void* workspace,
                                size_t workspace_bytes, int32_t draws, dpp_tune_entry* best,
                                void* stream) {
  clear_last_error();
  if (draws < 1 || draws > 4096)
    return set_last_error(DPP_ERR_INVALID_ARG, "dpp_autotune_batched: draws must be in [1, 4096]");
  if (batch < 1 || n_max < 1)
    return set_last_error(DPP_ERR_INVALID_ARG, "dpp_autotune_batched: empty batch");
  GpuId id;
  if (!gpu_id(&id)) return set_last_error(DPP_ERR_CUDA, "dpp_autotune_batched: no device");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int opts[2] = {128, 256};
  dpp_tune_entry win{};
  double win_sps = -1.0;
  dpp_status rs = DPP_OK;
  for (int i = 0; i < 2 && e == cudaSuccess && rs == DPP_OK; ++i) {
    dpp_tune_entry c{};
    c.op = kOpBatched;
    c.dtype = DPP_R64;
    c.precision = DPP_PREC_FP32;
    c.n_bucket = bucket_of(n_max);
    c.n = n_max;
    c.streams = 1;
    c.batched_threads = opts[i];
    tl_force = &c;
    auto draw = [&](uint64_t s) {
      return dpp_sample_batched(batch, n, K, ld, n_max, DPP_PREC_FP32, s, nullptr, keep, nullptr,
                                nullptr, results, workspace, workspace_bytes, stream);
    };
    rs = draw(seed + 1000000u);
    if (rs == DPP_OK) e = cudaEventRecord(e0, st);
    for (int d = 0; d < draws && rs == DPP_OK && e == cudaSuccess; ++d) rs = draw(seed + d);
    if (rs == DPP_OK && e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (rs == DPP_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    tl_force = nullptr;
    float ms = 0.f;
    if (rs == DPP_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rs == DPP_OK && e == cudaSuccess) {
      const double sps = ms > 0.f ? (double)batch * draws / (ms * 1e-3) : 0.0;
      if (sps > win_sps) {
        win_sps = sps;
        win = c;
        win.samples_per_s = sps;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rs != DPP_OK) return rs;
  if (e != cudaSuccess) return set_last_cuda_error(e, "dpp_autotune_batched");
  win.candidates = 2;
  put(id.name, id.sms, win);
  if (best) *best = win;
  return DPP_OK;
}

dpp_status dpp_tune_lookup(int32_t op, int64_t n, int32_t dtype, int32_t precision,
                           dpp_tune_entry* out) {
  clear_last_error();
  if (!out) return set_last_error(DPP_ERR_INVALID_ARG, "dpp_tune_lookup: out is NULL");
  if (!find(op, n, dtype, precision, out))
    return set_last_error(DPP_ERR_UNSUPPORTED, "dpp_tune_lookup: no entry for this key");
  return DPP_OK;
}

dpp_status dpp_tune_save(const char* path) {
  clear_last_error();
  if (!path) return set_last_error(DPP_ERR_INVALID_ARG, "dpp_tune_save: path is NULL");
  std::vector<Entry> copy;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    copy = g_table;
  }
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return set_last_error(DPP_ERR_INVALID_ARG, "dpp_tune_save: cannot open the file");
  fprintf(f, "{\"version\": 1, \"entries\": [");
  for (size_t i = 0; i < copy.size(); ++i) {
    const dpp_tune_entry& e = copy[i].e;
    std::string gpu;
    for (char ch : copy[i].gpu) {
      if (ch == '"' || ch == '\\') gpu.push_back('\\');
      gpu.push_back(ch);
    }
    fprintf(f,
            "%s\n  {\"gpu\": \"%s\", \"sms\": %d, \"op\": %d, \"dtype\": %d, \"precision\": %d, "
            "\"n_bucket\": %d, \"n\": %lld, \"outer_block\": %d, \"panel_pipeline\": %d, "
            "\"max_ctas\": %d, \"streams\": %d, \"samples_per_s\": %.6g, \"candidates\": %d, "
            "\"update_variant\": %d, \"batched_threads\": %d}",
            i ? "," : "", gpu.c_str(), copy[i].sms, e.op, e.dtype, e.precision, e.n_bucket,
            (long long)e.n, e.outer_block, e.panel_pipeline, e.max_ctas, e.streams,
            e.samples_per_s, e.candidates, e.update_variant, e.batched_threads);
  }
  fprintf(f, "\n]}\n");
  const bool ok = fclose(f) == 0;
  if (!ok || rename(tmp.c_str(), path) != 0)
    return set_last_error(DPP_ERR_INVALID_ARG, "dpp_tune_save: write failed");
  return DPP_OK;
}

dpp_status dpp_tune_load(const char* path) {
  clear_last_error();
  if (!path) return set_last_error(DPP_ERR_INVALID_ARG, "dpp_tune_load: path is NULL");
  std::string err;
  if (load_file(path, &err) < 0) {
    const std::string msg = "dpp_tune_load: " + err;
    return set_last_error(DPP_ERR_INVALID_ARG, msg.c_str());
  }
  return DPP_OK;
}

void dpp_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
}

}  // extern "C"
