// C ABI: context, argument checks, workspace, cached device layouts, and the
// five entry points of the sketched discord miner.
#include "tsk_internal.cuh"

#include <algorithm>
#include <array>
#include <cmath>
#include <chrono>
#include <cstdarg>
#include <cstring>
#include <thread>

int tsk_mp_pad();
int tsk_mp_chunk();
int tsk_mp_chunk_rows();

namespace {

// A small cache of immutable device blobs keyed by their host content, so that
// repeated calls with the same layout (and calls inside CUDA-graph capture)
// issue no host-to-device copies.
struct Blob {
  std::string key;
  void* dev = nullptr;
  size_t bytes = 0;
  std::vector<int64_t> meta;
  uint64_t stamp = 0;
};
struct BlobCache {
  std::vector<Blob> items;
  uint64_t clock = 0;
};
constexpr size_t kMaxBlobs = 16;

BlobCache& cache_of(tsk_ctx* ctx);

struct CtxExtra {
  BlobCache blobs;
};

}  // namespace

struct tsk_ctx_ext : tsk_ctx {
  CtxExtra extra;
};

namespace {
BlobCache& cache_of(tsk_ctx* ctx) { return static_cast<tsk_ctx_ext*>(ctx)->extra.blobs; }

bool capturing(tsk_ctx* ctx) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

template <typename T>
void append(std::string& k, const T* p, size_t n) {
  k.append(reinterpret_cast<const char*>(p), n * sizeof(T));
}

// Find or upload a blob.  `build` fills content and meta on a miss.
template <typename F>
const Blob* blob_get(tsk_ctx* ctx, const std::string& key, F&& build, tsk_status* st) {
  BlobCache& c = cache_of(ctx);
  for (auto& b : c.items)
    if (b.key == key) {
      b.stamp = ++c.clock;
      *st = TSK_OK;
      return &b;
    }
  if (capturing(ctx)) {
    *st = tsk_fail(ctx, TSK_ERR_UNSUPPORTED,
                   "layout not seen before capture: call once with the same layout before capturing a CUDA graph");
    return nullptr;
  }
  std::vector<char> content;
  std::vector<int64_t> meta;
  build(content, meta);
  if (c.items.size() >= kMaxBlobs) {
    auto it = std::min_element(c.items.begin(), c.items.end(),
                               [](const Blob& a, const Blob& b) { return a.stamp < b.stamp; });
    cudaStreamSynchronize(ctx->stream);
    cudaFree(it->dev);
    c.items.erase(it);
  }
  Blob b;
  b.key = key;
  b.bytes = std::max<size_t>(content.size(), 16);
  b.meta = std::move(meta);
  cudaError_t e = cudaMalloc(&b.dev, b.bytes);
  if (e != cudaSuccess) {
    *st = tsk_fail(ctx, TSK_ERR_OOM, "cudaMalloc(%zu) for layout: %s", b.bytes, cudaGetErrorString(e));
    return nullptr;
  }
  if (!content.empty()) {
    e = cudaMemcpy(b.dev, content.data(), content.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(b.dev);
      *st = tsk_cuda_fail(ctx, e, "cudaMemcpy(layout)");
      return nullptr;
    }
  }
  b.stamp = ++c.clock;
  c.items.push_back(std::move(b));
  *st = TSK_OK;
  return &c.items.back();
}

template <typename T>
size_t put(std::vector<char>& buf, const std::vector<T>& v) {
  size_t off = (buf.size() + 15) & ~size_t(15);
  buf.resize(off + v.size() * sizeof(T));
  if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

// Batch layout: per-series offsets plus the per-stream view used by the
// column statistics.  meta: [total_samples, sketch_blocks, off offsets...]
struct BatchLayout {
  const int64_t* cum;        // [n_series + 1]
  const int32_t* len;        // [n_series]
  const int64_t* blk_prefix; // [n_series + 1] 64-sample sketch blocks
  const int64_t* soff;       // [n_series * d + 1] stream offsets (d streams per series)
  const int32_t* slen;       // [n_series * d]
  int64_t total_samples;
  int64_t total_blocks;
};

tsk_status batch_layout(tsk_ctx* ctx, int32_t n_series, const int32_t* lens, int32_t d, BatchLayout* out) {
  std::string key = "batch";
  append(key, &n_series, 1);
  append(key, &d, 1);
  append(key, lens, n_series);
  tsk_status st = TSK_OK;
  const Blob* b = blob_get(ctx, key, [&](std::vector<char>& buf, std::vector<int64_t>& meta) {
    std::vector<int64_t> cum(n_series + 1, 0), blk(n_series + 1, 0), soff(static_cast<size_t>(n_series) * d + 1, 0);
    std::vector<int32_t> len(lens, lens + n_series), slen(static_cast<size_t>(n_series) * d);
    for (int s = 0; s < n_series; ++s) {
      cum[s + 1] = cum[s] + lens[s];
      blk[s + 1] = blk[s] + (lens[s] + 63) / 64;
      for (int j = 0; j < d; ++j) {
        const size_t q = static_cast<size_t>(s) * d + j;
        slen[q] = lens[s];
        soff[q + 1] = soff[q] + lens[s];
      }
    }
    meta = {cum[n_series], blk[n_series], 0, 0, 0, 0, 0};
    meta[2] = static_cast<int64_t>(put(buf, cum));
    meta[3] = static_cast<int64_t>(put(buf, len));
    meta[4] = static_cast<int64_t>(put(buf, blk));
    meta[5] = static_cast<int64_t>(put(buf, soff));
    meta[6] = static_cast<int64_t>(put(buf, slen));
  }, &st);
  if (!b) return st;
  char* base = static_cast<char*>(b->dev);
  out->total_samples = b->meta[0];
  out->total_blocks = b->meta[1];
  out->cum = reinterpret_cast<const int64_t*>(base + b->meta[2]);
  out->len = reinterpret_cast<const int32_t*>(base + b->meta[3]);
  out->blk_prefix = reinterpret_cast<const int64_t*>(base + b->meta[4]);
  out->soff = reinterpret_cast<const int64_t*>(base + b->meta[5]);
  out->slen = reinterpret_cast<const int32_t*>(base + b->meta[6]);
  return TSK_OK;
}

// Work units of one row stream against one column stream (the same stream for
// a self-join) on diagonals dmin, dmin+1, ...: bands of D diagonals, rows cut
// into units of H; rows where every diagonal of the band is valid go to
// `interior`, the band's last rows (diagonals running out, or the row side
// ending) to `tail` as one masked unit.
void add_units(int32_t q, int64_t l_row, int64_t l_col, int64_t dmin, int32_t H, int32_t D, int32_t chunk_rows,
               std::vector<int32_t>& interior, std::vector<int32_t>& tail) {
  for (int64_t d0 = dmin; d0 < l_col; d0 += D) {
    const int64_t rows = std::min(l_row, l_col - d0);                                 // rows with a cell
    int64_t rint = std::min(l_row, std::max<int64_t>(0, l_col - d0 - (D - 1)));       // rows with all D
    rint -= rint % chunk_rows;
    for (int64_t r0 = 0; r0 < rint; r0 += H) {
      const int64_t r1 = std::min<int64_t>(r0 + H, rint);
      interior.insert(interior.end(), {q, static_cast<int32_t>(d0), static_cast<int32_t>(r0), static_cast<int32_t>(r1)});
    }
    if (rows > rint)
      tail.insert(tail.end(), {q, static_cast<int32_t>(d0), static_cast<int32_t>(rint),
                               static_cast<int32_t>(static_cast<uint32_t>(rows) | 0x80000000u)});
  }
}

int32_t auto_rows(tsk_ctx* ctx, double cells) {
  // rows per work unit: about 64 units per resident warp, within [2048, 8192]
  // (warps claim runs of consecutive units, so small units cost few anchors)
  const int32_t D = tsk_mp_band_width();
  const double warps = static_cast<double>(ctx->sm_count) * 12.0;
  const double rows = cells / (warps * 64.0 * D);
  const int32_t step = tsk_mp_chunk_rows();
  int32_t H = static_cast<int32_t>(std::min(8192.0, std::max(2048.0, rows)));
  return (H + step - 1) / step * step;
}

tsk_status mp_plan(tsk_ctx* ctx, int32_t n, const int32_t* lens, const uint8_t* mask, int32_t m, int32_t excl,
                   int32_t prec, tsk_mp_plan* plan) {
  const int32_t D = tsk_mp_band_width();
  int32_t H = ctx->mp_H;
  if (H <= 0) {
    double cells = 0.0;
    for (int q = 0; q < n; ++q) {
      if (mask && !mask[q]) continue;
      const double e = static_cast<double>(lens[q]) - m + 1 - excl;
      if (e > 0) cells += e * (e + 1) / 2;
    }
    H = auto_rows(ctx, cells);
  }
  std::string key = "mp";
  const int32_t hdr[6] = {n, m, excl, prec, H, D};
  append(key, hdr, 6);
  append(key, lens, n);
  if (mask) append(key, mask, n);
  tsk_status st = TSK_OK;
  bool ntiles_overflow = false;
  const int pad = tsk_mp_pad();
  const int chunk = tsk_mp_chunk();
  const Blob* b = blob_get(ctx, key, [&](std::vector<char>& buf, std::vector<int64_t>& meta) {
    std::vector<int64_t> xoff(n + 1, 0), woff(n + 1, 0), chp(n + 1, 0), tp(n + 1, 0);
    std::vector<int32_t> len(lens, lens + n);
    std::vector<uint8_t> sm(n, 1);
    // float32 path: interior tiles of every band first, then the triangular ends
    // (the last rows of a band, where its diagonals run out, need masking)
    std::vector<int32_t> tiles_int, tiles_tri;
    const int32_t chunk_rows = tsk_mp_chunk_rows();
    for (int q = 0; q < n; ++q) {
      const bool on = !mask || mask[q];
      sm[q] = on ? 1 : 0;
      const int64_t l = static_cast<int64_t>(lens[q]) - m + 1;
      xoff[q + 1] = xoff[q] + lens[q];
      woff[q + 1] = woff[q] + ((l + pad + 3) & ~int64_t(3));
      chp[q + 1] = chp[q] + (on ? (l + chunk - 1) / chunk : 0);
      tp[q + 1] = tp[q] + ((on && prec == TSK_MP_FP64) ? std::max<int64_t>(0, l - excl) : 0);
      if (!on || prec == TSK_MP_FP64 || l <= excl) continue;
      add_units(q, l, l, excl, H, D, chunk_rows, tiles_int, tiles_tri);
    }
    tiles_int.insert(tiles_int.end(), tiles_tri.begin(), tiles_tri.end());
    const int64_t ntiles = prec == TSK_MP_FP64 ? tp[n] : static_cast<int64_t>(tiles_int.size() / 4);
    if (ntiles > 0x7fffffffLL) ntiles_overflow = true;
    meta.assign(11, 0);
    meta[0] = woff[n];
    meta[1] = chp[n];
    meta[2] = ntiles;
    meta[3] = xoff[n];
    meta[4] = static_cast<int64_t>(put(buf, xoff));
    meta[5] = static_cast<int64_t>(put(buf, len));
    meta[6] = static_cast<int64_t>(put(buf, sm));
    meta[7] = static_cast<int64_t>(put(buf, woff));
    meta[8] = static_cast<int64_t>(put(buf, chp));
    meta[9] = static_cast<int64_t>(put(buf, tp));
    meta[10] = static_cast<int64_t>(put(buf, tiles_int));
  }, &st);
  if (!b) return st;
  if (ntiles_overflow || b->meta[2] > 0x7fffffffLL)
    return tsk_fail(ctx, TSK_ERR_UNSUPPORTED, "mp_selfjoin: more than 2^31 work units; raise tsk_set_tile_rows");
  char* base = static_cast<char*>(b->dev);
  plan->m = m;
  plan->excl = excl;
  plan->H = H;
  plan->D = D;
  plan->prec = prec;
  plan->total_windows = b->meta[0];
  plan->total_chunks = b->meta[1];
  plan->total_tiles = b->meta[2];
  plan->total_samples = b->meta[3];
  plan->xoff = reinterpret_cast<int64_t*>(base + b->meta[4]);
  plan->len = reinterpret_cast<int32_t*>(base + b->meta[5]);
  plan->smask = reinterpret_cast<uint8_t*>(base + b->meta[6]);
  plan->woff = reinterpret_cast<int64_t*>(base + b->meta[7]);
  plan->chunk_prefix = reinterpret_cast<int64_t*>(base + b->meta[8]);
  plan->tile_prefix = reinterpret_cast<int64_t*>(base + b->meta[9]);
  plan->tiles = reinterpret_cast<int4*>(base + b->meta[10]);
  return TSK_OK;
}

// AB join: streams 0..n-1 are the test streams, n..2n-1 their training
// partners.  Test rows against training columns on diagonals >= 0, then
// training rows against test columns on diagonals >= 1.
tsk_status mp_plan_ab(tsk_ctx* ctx, int32_t n, const int32_t* len_a, const int32_t* len_b, int32_t m, int32_t prec,
                      tsk_mp_plan* plan) {
  const int32_t D = tsk_mp_band_width();
  int32_t H = ctx->mp_H;
  if (H <= 0) {
    double cells = 0.0;
    for (int q = 0; q < n; ++q) cells += static_cast<double>(len_a[q] - m + 1) * static_cast<double>(len_b[q] - m + 1);
    H = auto_rows(ctx, cells);
  }
  std::string key = "mpab";
  const int32_t hdr[5] = {n, m, H, D, prec};
  append(key, hdr, 5);
  append(key, len_a, n);
  append(key, len_b, n);
  tsk_status st = TSK_OK;
  const int pad = tsk_mp_pad();
  const int chunk = tsk_mp_chunk();
  const Blob* b = blob_get(ctx, key, [&](std::vector<char>& buf, std::vector<int64_t>& meta) {
    const int N = 2 * n;
    std::vector<int64_t> xoff(N + 1, 0), woff(N + 1, 0), chp(N + 1, 0), tp(N + 1, 0);
    std::vector<int32_t> len(N);
    std::vector<uint8_t> sm(N, 1);
    for (int q = 0; q < n; ++q) {
      len[q] = len_a[q];
      len[n + q] = len_b[q];
    }
    std::vector<int32_t> tiles_int, tiles_tri;
    const int32_t chunk_rows = tsk_mp_chunk_rows();
    for (int q = 0; q < N; ++q) {
      const int64_t l = static_cast<int64_t>(len[q]) - m + 1;
      const int p = q < n ? q + n : q - n;
      const int64_t lp = static_cast<int64_t>(len[p]) - m + 1;
      xoff[q + 1] = xoff[q] + len[q];
      woff[q + 1] = woff[q] + ((l + pad + 3) & ~int64_t(3));
      chp[q + 1] = chp[q] + (l + chunk - 1) / chunk;
      // float64 path: one thread per diagonal, diagonals 0.. (test rows) or 1.. (training rows)
      tp[q + 1] = tp[q] + (prec == TSK_MP_FP64 ? std::max<int64_t>(0, q < n ? lp : lp - 1) : 0);
    }
    if (prec != TSK_MP_FP64)
      for (int q = 0; q < N; ++q) {
        const int p = q < n ? q + n : q - n;
        add_units(q, static_cast<int64_t>(len[q]) - m + 1, static_cast<int64_t>(len[p]) - m + 1, q < n ? 0 : 1, H,
                  D, chunk_rows, tiles_int, tiles_tri);
      }
    tiles_int.insert(tiles_int.end(), tiles_tri.begin(), tiles_tri.end());
    meta.assign(11, 0);
    meta[0] = woff[N];
    meta[1] = chp[N];
    meta[2] = prec == TSK_MP_FP64 ? tp[N] : static_cast<int64_t>(tiles_int.size() / 4);
    meta[3] = xoff[N];
    meta[4] = static_cast<int64_t>(put(buf, xoff));
    meta[5] = static_cast<int64_t>(put(buf, len));
    meta[6] = static_cast<int64_t>(put(buf, sm));
    meta[7] = static_cast<int64_t>(put(buf, woff));
    meta[8] = static_cast<int64_t>(put(buf, chp));
    meta[9] = static_cast<int64_t>(put(buf, tp));
    meta[10] = static_cast<int64_t>(put(buf, tiles_int));
  }, &st);
  if (!b) return st;
  if (b->meta[2] > 0x7fffffffLL)
    return tsk_fail(ctx, TSK_ERR_UNSUPPORTED, "mp_abjoin: more than 2^31 work units; raise tsk_set_tile_rows");
  char* base = static_cast<char*>(b->dev);
  plan->m = m;
  plan->excl = 0;
  plan->H = H;
  plan->D = D;
  plan->prec = prec;
  plan->total_windows = b->meta[0];
  plan->total_chunks = b->meta[1];
  plan->total_tiles = b->meta[2];
  plan->total_samples = b->meta[3];
  plan->xoff = reinterpret_cast<int64_t*>(base + b->meta[4]);
  plan->len = reinterpret_cast<int32_t*>(base + b->meta[5]);
  plan->smask = reinterpret_cast<uint8_t*>(base + b->meta[6]);
  plan->woff = reinterpret_cast<int64_t*>(base + b->meta[7]);
  plan->chunk_prefix = reinterpret_cast<int64_t*>(base + b->meta[8]);
  plan->tile_prefix = reinterpret_cast<int64_t*>(base + b->meta[9]);
  plan->tiles = reinterpret_cast<int4*>(base + b->meta[10]);
  return TSK_OK;
}

tsk_status enter(tsk_ctx* ctx) {
  if (!ctx) return TSK_ERR_INVALID_ARG;
  ctx->last_error.clear();
  const cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return tsk_cuda_fail(ctx, e, "cudaSetDevice");
  return TSK_OK;
}

tsk_status check_lens(tsk_ctx* ctx, int32_t n, const int32_t* lens, int32_t min_len, const char* what) {
  if (!lens) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "%s: length array is NULL", what);
  for (int32_t q = 0; q < n; ++q)
    if (lens[q] < min_len)
      return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "%s: length[%d] = %d is below the minimum %d", what, q, lens[q], min_len);
  return TSK_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// shared host helpers
// ---------------------------------------------------------------------------
tsk_status tsk_fail(tsk_ctx* ctx, tsk_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return st;
}

tsk_status tsk_cuda_fail(tsk_ctx* ctx, cudaError_t e, const char* where) {
  return tsk_fail(ctx, e == cudaErrorMemoryAllocation ? TSK_ERR_OOM : TSK_ERR_CUDA, "%s: %s (%s)", where,
                  cudaGetErrorString(e), cudaGetErrorName(e));
}

tsk_status tsk_ws_require(tsk_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return TSK_OK;
  if (capturing(ctx))
    return tsk_fail(ctx, TSK_ERR_OOM, "workspace needs %zu bytes but holds %zu: call tsk_reserve before capture", bytes,
                    ctx->ws_bytes);
  if (ctx->ws) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  const size_t want = bytes + bytes / 4 + (1u << 20);
  cudaError_t e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return tsk_fail(ctx, TSK_ERR_OOM, "workspace cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
  }
  ctx->ws_bytes = want;
  return TSK_OK;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" TSK_API tsk_status tsk_create(tsk_ctx** out, int32_t device, void* cuda_stream) {
  if (!out) return TSK_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return TSK_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return TSK_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return TSK_ERR_CUDA;
  auto* ctx = new tsk_ctx_ext();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return TSK_ERR_CUDA;
  }
  ctx->sm_count = prop.multiProcessorCount;
  if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
    delete ctx;
    return TSK_ERR_OOM;
  }
  *out = ctx;
  return TSK_OK;
}

extern "C" TSK_API tsk_status tsk_set_stream(tsk_ctx* ctx, void* cuda_stream) {
  if (!ctx) return TSK_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return TSK_OK;
}

extern "C" TSK_API void tsk_destroy(tsk_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& b : cache_of(ctx).items) cudaFree(b.dev);
  for (auto& ev : ctx->prof_events)
    for (auto& pr : ev) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_err) cudaFree(ctx->d_err);
  delete static_cast<tsk_ctx_ext*>(ctx);
}

extern "C" TSK_API const char* tsk_last_error(const tsk_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

extern "C" TSK_API tsk_status tsk_reserve(tsk_ctx* ctx, size_t bytes) {
  tsk_status st = enter(ctx);
  if (st) return st;
  return tsk_ws_require(ctx, bytes);
}

tsk_prof_scope::tsk_prof_scope(tsk_ctx* c, int k) : ctx(c), kernel(k) {
  if (!ctx->prof || capturing(ctx)) return;
  if (cudaEventCreate(&e1) != cudaSuccess || cudaEventCreate(&e2) != cudaSuccess) {
    cudaGetLastError();
    e1 = e2 = nullptr;
    return;
  }
  cudaEventRecord(e1, ctx->stream);
}

tsk_prof_scope::~tsk_prof_scope() {
  if (!e1) return;
  cudaEventRecord(e2, ctx->stream);
  ctx->prof_events[kernel].emplace_back(e1, e2);
}

extern "C" TSK_API tsk_status tsk_profile_enable(tsk_ctx* ctx, int32_t enable) {
  if (!ctx) return TSK_ERR_INVALID_ARG;
  ctx->prof = enable != 0;
  return TSK_OK;
}

extern "C" TSK_API tsk_status tsk_profile_read(tsk_ctx* ctx, int32_t kernel, double* total_ms, int64_t* launches) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (kernel < 0 || kernel >= TSK_PROF_COUNT || !total_ms || !launches)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "tsk_profile_read: bad arguments");
  double sum = 0.0;
  auto& ev = ctx->prof_events[kernel];
  for (auto& pr : ev) {
    TSK_CUDA_TRY(ctx, cudaEventSynchronize(pr.second));
    float ms = 0.f;
    TSK_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, pr.first, pr.second));
    sum += ms;
  }
  *total_ms = sum;
  *launches = static_cast<int64_t>(ev.size());
  for (auto& pr : ev) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  ev.clear();
  return TSK_OK;
}

extern "C" TSK_API tsk_status tsk_set_tile_rows(tsk_ctx* ctx, int32_t rows) {
  if (!ctx) return TSK_ERR_INVALID_ARG;
  if (rows != 0 && (rows < 32 || rows > (1 << 20) || rows % 32 != 0))
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "tsk_set_tile_rows: rows must be 0 (automatic) or a multiple of 32 in [32, 2^20]");
  ctx->mp_H = rows;
  return TSK_OK;
}

extern "C" TSK_API int64_t tsk_launch_count(const tsk_ctx* ctx) { return ctx ? ctx->launches : -1; }

extern "C" TSK_API tsk_status tsk_selftest_timeout(tsk_ctx* ctx) {
  tsk_status st = enter(ctx);
  if (st) return st;
  return tsk_launch_selftest_wait(ctx);
}

extern "C" TSK_API tsk_status tsk_sync(tsk_ctx* ctx, double timeout_s) {
  tsk_status st = enter(ctx);
  if (st) return st;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(ctx->stream);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return tsk_cuda_fail(ctx, e, "stream");
    if (timeout_s > 0) {
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > timeout_s) return tsk_fail(ctx, TSK_ERR_TIMEOUT, "stream still busy after %.3f s", el);
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  int flag = 0;
  TSK_CUDA_TRY(ctx, cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    TSK_CUDA_TRY(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
    if (flag & TSK_DEVERR_NONFINITE) return tsk_fail(ctx, TSK_ERR_NONFINITE, "non-finite value in an input series");
    if (flag & TSK_DEVERR_TIMEOUT) return tsk_fail(ctx, TSK_ERR_TIMEOUT, "a device-side wait gave up (results invalid)");
  }
  return TSK_OK;
}

extern "C" TSK_API tsk_status tsk_mp_workspace_bytes(tsk_ctx* ctx, int32_t n_streams, const int32_t* stream_len_host,
                                                     int32_t m, size_t* bytes_out) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (!bytes_out || n_streams < 1 || m < 2) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "bad arguments");
  if ((st = check_lens(ctx, n_streams, stream_len_host, m, "tsk_mp_workspace_bytes"))) return st;
  tsk_mp_plan plan;
  plan.prec = TSK_MP_FP32;
  const int pad = tsk_mp_pad();
  int64_t W = 0;
  for (int q = 0; q < n_streams; ++q) W += ((static_cast<int64_t>(stream_len_host[q]) - m + 1 + pad + 3) & ~int64_t(3));
  plan.total_windows = W;
  *bytes_out = std::max(tsk_mp_ws_bytes(plan, n_streams), static_cast<size_t>(0));
  plan.prec = TSK_MP_FP64;
  *bytes_out = std::max(*bytes_out, tsk_mp_ws_bytes(plan, n_streams));
  return TSK_OK;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
extern "C" TSK_API tsk_status ts_sketch_build(tsk_ctx* ctx, const void* T, int32_t t_dtype, int32_t n_series,
                                              const int32_t* series_len_host, int32_t d, const float* R, int32_t k,
                                              int32_t precision, void* S, double* stats) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (!T || !R || !S) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_build: T, R and S must be non-NULL");
  if (t_dtype != TSK_F32 && t_dtype != TSK_F64) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_build: bad t_dtype");
  if (precision < TSK_SKETCH_BF16 || precision > TSK_SKETCH_FP64)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_build: bad precision");
  if (n_series < 1 || d < 1 || k < 1 || k > 4096)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_build: need n_series >= 1, d >= 1, 1 <= k <= 4096");
  if ((st = check_lens(ctx, n_series, series_len_host, 1, "ts_sketch_build"))) return st;
  BatchLayout L{};
  if ((st = batch_layout(ctx, n_series, series_len_host, d, &L))) return st;
  const size_t stat_bytes = stats ? 0 : tsk_carver::bytes_for(static_cast<size_t>(n_series) * d * 2, 8);
  const size_t sk_bytes = precision == TSK_SKETCH_BF16
                              ? tsk_sketch_ws_bytes(n_series, d, k, L.total_blocks, L.total_samples, ctx->sm_count)
                              : 0;
  if ((st = tsk_ws_require(ctx, stat_bytes + sk_bytes))) return st;
  tsk_carver cv(ctx->ws);
  double* stv = stats ? stats : cv.take<double>(static_cast<size_t>(n_series) * d * 2);
  char* skws = cv.take<char>(sk_bytes > 0 ? sk_bytes : 1);
  if ((st = tsk_launch_colstats(ctx, T, t_dtype, L.soff, L.slen, static_cast<int64_t>(n_series) * d, stv))) return st;
  return tsk_launch_sketch(ctx, T, t_dtype, n_series, L.cum, L.len, L.blk_prefix, L.total_blocks, d, R, k, precision,
                           stv, S, L.total_samples, skws);
}

extern "C" TSK_API tsk_status ts_sketch_update_dims(tsk_ctx* ctx, void* S, const void* T_dims, int32_t t_dtype,
                                                    int32_t n_series, const int32_t* series_len_host, int32_t nd,
                                                    const float* R_rows_host, const int8_t* op_host, int32_t k,
                                                    int32_t precision, double* stats, uint8_t* dirty_host) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (!S || !T_dims || !R_rows_host || !op_host)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_update_dims: S, T_dims, R_rows_host, op_host must be non-NULL");
  if (t_dtype != TSK_F32 && t_dtype != TSK_F64) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "bad t_dtype");
  if (precision < TSK_SKETCH_BF16 || precision > TSK_SKETCH_FP64) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "bad precision");
  if (n_series < 1 || nd < 1 || k < 1 || k > 4096)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_update_dims: need n_series >= 1, nd >= 1, 1 <= k <= 4096");
  for (int q = 0; q < nd; ++q)
    if (op_host[q] != 1 && op_host[q] != -1)
      return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_update_dims: op[%d] must be +1 or -1", q);
  if ((st = check_lens(ctx, n_series, series_len_host, 1, "ts_sketch_update_dims"))) return st;
  BatchLayout L{};
  if ((st = batch_layout(ctx, n_series, series_len_host, nd, &L))) return st;
  const size_t nstat = static_cast<size_t>(n_series) * nd * 2;
  if ((st = tsk_ws_require(ctx, tsk_carver::bytes_for(nstat, 8)))) return st;
  tsk_carver cv(ctx->ws);
  double* stv = cv.take<double>(nstat);
  // the projection rows and signs go through the layout cache (no copy when a
  // call with the same rows was made before, e.g. before graph capture)
  std::string key = "upd";
  append(key, &nd, 1);
  append(key, &k, 1);
  append(key, R_rows_host, static_cast<size_t>(nd) * k);
  append(key, op_host, nd);
  const Blob* ub = blob_get(ctx, key, [&](std::vector<char>& buf, std::vector<int64_t>& meta) {
    std::vector<float> rr(R_rows_host, R_rows_host + static_cast<size_t>(nd) * k);
    std::vector<int8_t> oo(op_host, op_host + nd);
    meta = {static_cast<int64_t>(put(buf, rr)), static_cast<int64_t>(put(buf, oo))};
  }, &st);
  if (!ub) return st;
  const float* d_R = reinterpret_cast<const float*>(static_cast<char*>(ub->dev) + ub->meta[0]);
  const int8_t* d_op = reinterpret_cast<const int8_t*>(static_cast<char*>(ub->dev) + ub->meta[1]);
  if ((st = tsk_launch_colstats(ctx, T_dims, t_dtype, L.soff, L.slen, static_cast<int64_t>(n_series) * nd, stv))) return st;
  if ((st = tsk_launch_update_dims(ctx, S, T_dims, t_dtype, n_series, L.cum, L.len, L.total_samples, nd, d_R, d_op, k,
                                   precision, stv)))
    return st;
  if (stats)
    TSK_CUDA_TRY(ctx, cudaMemcpyAsync(stats, stv, sizeof(double) * nstat, cudaMemcpyDeviceToDevice, ctx->stream));
  if (dirty_host)
    for (int g = 0; g < k; ++g) {
      uint8_t f = 0;
      for (int q = 0; q < nd; ++q) f |= (R_rows_host[q * k + g] != 0.f) ? 1 : 0;
      dirty_host[g] = f;
    }
  return TSK_OK;
}

extern "C" TSK_API tsk_status ts_sketch_point_update(tsk_ctx* ctx, void* S, void* T, int32_t t_dtype,
                                                     int32_t n_series, const int32_t* series_len_host, int32_t d,
                                                     const float* R, int32_t k, int32_t precision, const double* stats,
                                                     int32_t n_upd, const int32_t* upd_series_host,
                                                     const int32_t* upd_dim_host, const int32_t* upd_time_host,
                                                     const double* upd_delta_host) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (!S || !R || !stats) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_point_update: S, R, stats must be non-NULL");
  if (t_dtype != TSK_F32 && t_dtype != TSK_F64) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "bad t_dtype");
  if (precision < TSK_SKETCH_BF16 || precision > TSK_SKETCH_FP64) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "bad precision");
  if (precision == TSK_SKETCH_BF16 && !T)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_point_update: the bf16-matched sketch needs T (old samples)");
  if (n_series < 1 || d < 1 || k < 1 || n_upd < 0)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_point_update: need n_series, d, k >= 1 and n_upd >= 0");
  if (n_upd == 0) return TSK_OK;
  if (!upd_series_host || !upd_dim_host || !upd_time_host || !upd_delta_host)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_point_update: update arrays must be non-NULL");
  if ((st = check_lens(ctx, n_series, series_len_host, 1, "ts_sketch_point_update"))) return st;
  // distinct points, deltas of repeated points summed in the given order
  std::vector<std::pair<std::array<int32_t, 3>, double>> pts;
  pts.reserve(n_upd);
  for (int32_t u = 0; u < n_upd; ++u) {
    const int32_t s = upd_series_host[u], j = upd_dim_host[u], t = upd_time_host[u];
    if (s < 0 || s >= n_series || j < 0 || j >= d || t < 0 || t >= series_len_host[s])
      return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_point_update: update %d (%d, %d, %d) out of range", u, s, j, t);
    if (!std::isfinite(upd_delta_host[u]))
      return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "ts_sketch_point_update: delta %d is not finite", u);
    pts.push_back({{s, j, t}, upd_delta_host[u]});
  }
  std::stable_sort(pts.begin(), pts.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  std::vector<int4> up;
  std::vector<double> dl;
  for (size_t u = 0; u < pts.size(); ++u) {
    if (!up.empty() && up.back().x == pts[u].first[0] && up.back().y == pts[u].first[1] &&
        up.back().z == pts[u].first[2]) {
      dl.back() += pts[u].second;
    } else {
      up.push_back(make_int4(pts[u].first[0], pts[u].first[1], pts[u].first[2], 0));
      dl.push_back(pts[u].second);
    }
  }
  BatchLayout L{};
  if ((st = batch_layout(ctx, n_series, series_len_host, d, &L))) return st;
  const size_t np = up.size();
  if ((st = tsk_ws_require(ctx, tsk_carver::bytes_for(np, sizeof(int4)) + tsk_carver::bytes_for(np, 8)))) return st;
  tsk_carver cv(ctx->ws);
  int4* d_pts = cv.take<int4>(np);
  double* d_dl = cv.take<double>(np);
  TSK_CUDA_TRY(ctx, cudaMemcpyAsync(d_pts, up.data(), sizeof(int4) * np, cudaMemcpyHostToDevice, ctx->stream));
  TSK_CUDA_TRY(ctx, cudaMemcpyAsync(d_dl, dl.data(), sizeof(double) * np, cudaMemcpyHostToDevice, ctx->stream));
  // (copies from pageable memory return once staged, so the vectors may go out of scope)
  return tsk_launch_point_update(ctx, S, T, t_dtype, d_pts, d_dl, static_cast<int32_t>(np), L.cum, L.len, d, R, k,
                                 precision, stats);
}

extern "C" TSK_API tsk_status mp_selfjoin(tsk_ctx* ctx, const void* X, int32_t x_dtype, int32_t n_streams,
                                          const int32_t* stream_len_host, const uint8_t* stream_mask_host, int32_t m,
                                          int32_t excl, int32_t precision, void* P, int32_t* I) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (!X || !P || !I) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin: X, P and I must be non-NULL");
  if (x_dtype != TSK_F32 && x_dtype != TSK_F64) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin: bad x_dtype");
  if (precision != TSK_MP_FP32 && precision != TSK_MP_FP64)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin: bad precision");
  if (n_streams < 1) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin: n_streams must be >= 1");
  if (m < 2 || m > 4096) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin: need 2 <= m <= 4096 (got %d)", m);
  if (excl < 1) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin: excl must be >= 1");
  if ((st = check_lens(ctx, n_streams, stream_len_host, m, "mp_selfjoin"))) return st;
  tsk_mp_plan plan;
  if ((st = mp_plan(ctx, n_streams, stream_len_host, stream_mask_host, m, excl, precision, &plan))) return st;
  if ((st = tsk_ws_require(ctx, tsk_mp_ws_bytes(plan, n_streams)))) return st;
  return tsk_run_mp(ctx, X, x_dtype, n_streams, plan, m, excl, precision, P, I, static_cast<char*>(ctx->ws));
}

extern "C" TSK_API tsk_status mp_selfjoin_update(tsk_ctx* ctx, const float* X, int32_t n_streams,
                                                 const int32_t* stream_len_host, int32_t m, int32_t excl, float* P,
                                                 int32_t* I, int32_t n_pts, const int32_t* pt_stream_host,
                                                 const int32_t* pt_time_host) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (!X || !P || !I) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin_update: X, P and I must be non-NULL");
  if (n_streams < 1) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin_update: n_streams must be >= 1");
  if (m < 2 || m > 4096) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin_update: need 2 <= m <= 4096 (got %d)", m);
  if (excl < 1) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin_update: excl must be >= 1");
  if (n_pts < 0) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin_update: n_pts must be >= 0");
  if ((st = check_lens(ctx, n_streams, stream_len_host, m, "mp_selfjoin_update"))) return st;
  if (n_pts == 0) return TSK_OK;
  if (!pt_stream_host || !pt_time_host)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin_update: point arrays must be non-NULL");
  // affected windows of every point: t - m + 1 .. t, merged into sorted runs per stream
  std::vector<std::pair<int32_t, int32_t>> iv;
  iv.reserve(n_pts);
  for (int32_t u = 0; u < n_pts; ++u) {
    const int32_t q = pt_stream_host[u], t = pt_time_host[u];
    if (q < 0 || q >= n_streams || t < 0 || t >= stream_len_host[q])
      return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_selfjoin_update: point %d (%d, %d) out of range", u, q, t);
    iv.push_back({q, t});
  }
  std::sort(iv.begin(), iv.end());
  std::vector<int4> runs;
  std::vector<uint8_t> mask(n_streams, 0);
  size_t tiles_max = 0;
  for (const auto& p : iv) {
    const int32_t q = p.first;
    const int32_t l = stream_len_host[q] - m + 1;
    const int32_t a = std::max(0, p.second - m + 1), b = std::min(l, p.second + 1);
    if (a >= b) continue;
    mask[q] = 1;
    if (!runs.empty() && runs.back().x == q && a <= runs.back().z) {
      runs.back().z = std::max(runs.back().z, b);
    } else {
      runs.push_back(make_int4(q, a, b, 0));
      tiles_max += 2 * static_cast<size_t>((std::max(0, l - excl) + tsk_mp_band_width() - 1) / tsk_mp_band_width());
    }
  }
  if (runs.empty()) return TSK_OK;
  tsk_mp_plan plan;
  if ((st = mp_plan(ctx, n_streams, stream_len_host, mask.data(), m, excl, TSK_MP_FP32, &plan))) return st;
  // Re-scanning a changed window's neighbours costs about 1/64 of a whole
  // profile per window of A (measured on GB300: break-even near 1.5% of the
  // windows changed); past that the touched streams are profiled whole.
  int64_t changed = 0, windows = 0;
  for (const int4& u : runs) changed += u.z - u.y;
  for (int32_t q = 0; q < n_streams; ++q)
    if (mask[q]) windows += stream_len_host[q] - m + 1;
  if (changed * 64 > windows) {
    if ((st = tsk_ws_require(ctx, tsk_mp_ws_bytes(plan, n_streams)))) return st;
    return tsk_run_mp(ctx, X, TSK_F32, n_streams, plan, m, excl, TSK_MP_FP32, P, I, static_cast<char*>(ctx->ws));
  }
  if ((st = tsk_ws_require(ctx, tsk_mp_update_ws_bytes(plan, n_streams, runs.size(), tiles_max)))) return st;
  return tsk_run_mp_update(ctx, X, n_streams, stream_len_host, plan, m, excl, P, I, runs, static_cast<char*>(ctx->ws));
}

extern "C" TSK_API tsk_status mp_abjoin(tsk_ctx* ctx, const void* A, const void* B, int32_t x_dtype, int32_t n_pairs,
                                        const int32_t* len_a_host, const int32_t* len_b_host, int32_t m,
                                        int32_t precision, void* P_a, int32_t* I_a, void* P_b, int32_t* I_b) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (!A || !B || !P_a || !I_a) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_abjoin: A, B, P_a and I_a must be non-NULL");
  if ((P_b == nullptr) != (I_b == nullptr))
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_abjoin: P_b and I_b must be both NULL or both non-NULL");
  if (x_dtype != TSK_F32 && x_dtype != TSK_F64) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_abjoin: bad x_dtype");
  if (precision != TSK_MP_FP32 && precision != TSK_MP_FP64)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_abjoin: bad precision");
  if (n_pairs < 1) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_abjoin: n_pairs must be >= 1");
  if (m < 2 || m > 4096) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_abjoin: need 2 <= m <= 4096 (got %d)", m);
  if ((st = check_lens(ctx, n_pairs, len_a_host, m, "mp_abjoin (test)"))) return st;
  if ((st = check_lens(ctx, n_pairs, len_b_host, m, "mp_abjoin (train)"))) return st;
  tsk_mp_plan plan;
  if ((st = mp_plan_ab(ctx, n_pairs, len_a_host, len_b_host, m, precision, &plan))) return st;
  if ((st = tsk_ws_require(ctx, tsk_mp_ws_bytes(plan, 2 * n_pairs)))) return st;
  return tsk_run_mp_ab(ctx, A, B, x_dtype, n_pairs, plan, m, precision, P_a, I_a, P_b, I_b,
                       static_cast<char*>(ctx->ws));
}

extern "C" TSK_API tsk_status discord_topk(tsk_ctx* ctx, const void* P, int32_t p_dtype, const int32_t* I,
                                           int32_t n_series, const int32_t* series_len_host, int32_t group, int32_t m,
                                           int32_t K, int32_t topk_excl, int32_t* idx, int32_t* grp, void* score,
                                           int32_t* nn) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (!P || !I || !idx || !grp || !score || !nn)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "discord_topk: array arguments must be non-NULL");
  if (p_dtype != TSK_F32 && p_dtype != TSK_F64) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "discord_topk: bad p_dtype");
  if (n_series < 1 || group < 1 || K < 1 || topk_excl < 1 || m < 1)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "discord_topk: need n_series, group, K, topk_excl, m >= 1");
  if ((st = check_lens(ctx, n_series, series_len_host, m, "discord_topk"))) return st;
  BatchLayout L{};
  if ((st = batch_layout(ctx, n_series, series_len_host, 1, &L))) return st;
  const size_t need = tsk_carver::bytes_for(L.total_samples, 4) + tsk_carver::bytes_for(L.total_samples, 8);
  if ((st = tsk_ws_require(ctx, need))) return st;
  return tsk_launch_topk(ctx, P, p_dtype, I, n_series, L.cum, L.len, group, m, K, topk_excl, idx, grp, score, nn,
                         static_cast<char*>(ctx->ws), L.total_samples);
}

extern "C" TSK_API tsk_status dimension_detection(tsk_ctx* ctx, const void* T, int32_t t_dtype, int32_t n_series,
                                                  const int32_t* series_len_host, int32_t d, const float* R,
                                                  int32_t k, int32_t m, int32_t excl, int32_t K, const int32_t* idx,
                                                  const int32_t* grp, int32_t* dim, double* dim_score,
                                                  int32_t* dim_nn, double* dim_scores, void* T_sel,
                                                  const void* T_train, const int32_t* train_len_host,
                                                  void* T_sel_train) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (!T || !R || !idx || !grp || !dim || !dim_score || !dim_nn)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "dimension_detection: required arrays must be non-NULL");
  if (t_dtype != TSK_F32 && t_dtype != TSK_F64)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "dimension_detection: bad t_dtype");
  if (n_series < 1 || d < 1 || k < 1 || K < 1)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "dimension_detection: need n_series, d, k, K >= 1");
  if (m < 2 || m > 4096)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "dimension_detection: need 2 <= m <= 4096 (got %d)", m);
  const bool ab = T_train != nullptr;
  if (ab && !train_len_host)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "dimension_detection: T_train needs train_len_host");
  if (!ab && T_sel_train)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "dimension_detection: T_sel_train needs T_train");
  if (!ab && excl < 1) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "dimension_detection: excl must be >= 1");
  if ((st = check_lens(ctx, n_series, series_len_host, m, "dimension_detection"))) return st;
  if (ab && (st = check_lens(ctx, n_series, train_len_host, m, "dimension_detection (train)"))) return st;
  BatchLayout L{}, Lt{};
  if ((st = batch_layout(ctx, n_series, series_len_host, d, &L))) return st;
  const int32_t* scan_len = ab ? train_len_host : series_len_host;
  if (ab && (st = batch_layout(ctx, n_series, train_len_host, d, &Lt))) return st;
  if (!ab) Lt = L;
  // scan items: (stream, chunk of windows) per series of the scanned side
  std::string key = "dims";
  const int32_t hdr[3] = {n_series, d, static_cast<int32_t>(tsk_dims_window_chunk())};
  append(key, hdr, 3);
  append(key, &m, 1);
  append(key, scan_len, n_series);
  const int64_t W = tsk_dims_window_chunk();
  const Blob* b = blob_get(ctx, key, [&](std::vector<char>& buf, std::vector<int64_t>& meta) {
    std::vector<int64_t> pre(static_cast<size_t>(n_series) + 1, 0);
    for (int s = 0; s < n_series; ++s) {
      const int64_t l = static_cast<int64_t>(scan_len[s]) - m + 1;
      pre[s + 1] = pre[s] + static_cast<int64_t>(d) * ((l + W - 1) / W);
    }
    meta = {pre[n_series], 0};
    meta[1] = static_cast<int64_t>(put(buf, pre));
  }, &st);
  if (!b) return st;
  const int64_t total_items = b->meta[0];
  const int64_t* item_prefix = reinterpret_cast<const int64_t*>(static_cast<char*>(b->dev) + b->meta[1]);
  if ((st = tsk_ws_require(ctx, tsk_dims_ws_bytes(n_series, K, d, m)))) return st;
  return tsk_launch_dims(ctx, T, ab ? T_train : T, t_dtype, n_series, L.cum, L.len, Lt.cum, Lt.len, item_prefix,
                         total_items, L.total_samples, Lt.total_samples, d, R, k, m, ab ? 0 : excl, K, idx, grp, dim,
                         dim_score, dim_nn, dim_scores, T_sel, ab ? T_sel_train : nullptr,
                         static_cast<char*>(ctx->ws));
}

extern "C" TSK_API tsk_status mp_backward(tsk_ctx* ctx, const float* dscore, const int32_t* idx, const int32_t* grp,
                                          const int32_t* nn, int32_t K, const void* T, int32_t t_dtype,
                                          const double* stats, const float* R, const float* S, int32_t n_series,
                                          const int32_t* series_len_host, int32_t d, int32_t k, int32_t m, float* dT,
                                          float* dR) {
  tsk_status st = enter(ctx);
  if (st) return st;
  if (!dscore || !idx || !grp || !nn || !T || !stats || !R || !S || !dT || !dR)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_backward: array arguments must be non-NULL");
  if (t_dtype != TSK_F32 && t_dtype != TSK_F64) return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_backward: bad t_dtype");
  if (n_series < 1 || K < 1 || d < 1 || k < 1 || k > 4096 || m < 2)
    return tsk_fail(ctx, TSK_ERR_INVALID_ARG, "mp_backward: need n_series, K, d >= 1, 1 <= k <= 4096, m >= 2");
  if ((st = check_lens(ctx, n_series, series_len_host, m, "mp_backward"))) return st;
  BatchLayout L{};
  if ((st = batch_layout(ctx, n_series, series_len_host, d, &L))) return st;
  const int64_t nsel = static_cast<int64_t>(n_series) * K;
  const size_t need = tsk_carver::bytes_for(static_cast<size_t>(nsel) * 2 * m, 4) +
                      tsk_carver::bytes_for(static_cast<size_t>(n_series) * d * 2, 8);
  if ((st = tsk_ws_require(ctx, need))) return st;
  int32_t max_len = 0;
  for (int32_t q = 0; q < n_series; ++q) max_len = std::max(max_len, series_len_host[q]);
  return tsk_launch_backward(ctx, dscore, idx, grp, nn, K, T, t_dtype, stats, R, S, n_series, L.cum, L.len,
                             max_len, d, k, m, dT, dR, static_cast<char*>(ctx->ws));
}
