// Checkpoint files (host code only; no counterpart in the paper): arrays of
// the sketch family (S, W, a refiner's dS) and the learned refiner's state,
// so that a long SGD run on the IVY loss (Eq. 2.1) can stop and resume.
//
// Every number is written byte by byte in little-endian order, whatever the
// host's order, so a file moves between machines.  A file is written to
// "<path>.tmp" and renamed over path once complete, so a crash mid-write
// never leaves a truncated checkpoint under the real name.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tsk.h"
#include "tsk_internal.cuh"

using tsk::set_thread_error;

namespace {

constexpr char kArrMagic[8] = {'T', 'S', 'K', 'A', 'R', 'R', '1', '\0'};
constexpr char kRefMagic[8] = {'T', 'S', 'K', 'R', 'E', 'F', '1', '\0'};
constexpr int kArrHeader = 32;
constexpr int kRefHeader = 72;

size_t elt_size(int prec) {
  return prec == TSK_FP64 ? 8 : prec == TSK_FP32 ? 4 : prec == TSK_BF16 ? 2 : 0;
}

bool host_little() {
  const uint16_t one = 1;
  unsigned char b;
  memcpy(&b, &one, 1);
  return b == 1;
}

void put_u32(unsigned char* p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = (unsigned char)(v >> (8 * i));
}
void put_u64(unsigned char* p, uint64_t v) {
  for (int i = 0; i < 8; ++i) p[i] = (unsigned char)(v >> (8 * i));
}
uint32_t get_u32(const unsigned char* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
uint64_t get_u64(const unsigned char* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}
void put_f64(unsigned char* p, double x) {
  uint64_t v;
  memcpy(&v, &x, 8);
  put_u64(p, v);
}
double get_f64(const unsigned char* p) {
  const uint64_t v = get_u64(p);
  double x;
  memcpy(&x, &v, 8);
  return x;
}

// count elements of es bytes each, host order -> little-endian in the file
bool write_elems(FILE* f, const void* src, size_t count, size_t es) {
  if (count == 0) return true;
  if (host_little()) return fwrite(src, es, count, f) == count;
  const unsigned char* s = (const unsigned char*)src;
  std::vector<unsigned char> buf(es * 4096);
  for (size_t i = 0; i < count;) {
    const size_t c = count - i < 4096 ? count - i : 4096;
    for (size_t e = 0; e < c; ++e)
      for (size_t b = 0; b < es; ++b) buf[e * es + b] = s[(i + e) * es + (es - 1 - b)];
    if (fwrite(buf.data(), es, c, f) != c) return false;
    i += c;
  }
  return true;
}

bool read_elems(FILE* f, void* dst, size_t count, size_t es) {
  if (count == 0) return true;
  if (fread(dst, es, count, f) != count) return false;
  if (!host_little()) {
    unsigned char* d = (unsigned char*)dst;
    for (size_t e = 0; e < count; ++e)
      for (size_t b = 0; b < es / 2; ++b) {
        const unsigned char t = d[e * es + b];
        d[e * es + b] = d[e * es + es - 1 - b];
        d[e * es + es - 1 - b] = t;
      }
  }
  return true;
}

// Writes header + payloads to path.tmp, then renames it over path.
tsk_status write_file(const char* fn, const char* path, const unsigned char* hdr, size_t hlen,
                      const void* const* data, const size_t* counts, int nparts, size_t es) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) {
    set_thread_error("%s: cannot open %s for writing", fn, tmp.c_str());
    return TSK_EINVAL;
  }
  bool ok = fwrite(hdr, 1, hlen, f) == hlen;
  for (int i = 0; ok && i < nparts; ++i) ok = write_elems(f, data[i], counts[i], es);
  ok = (fflush(f) == 0) && ok;
  ok = (fclose(f) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    set_thread_error("%s: writing %s failed", fn, path);
    return TSK_EINVAL;
  }
  return TSK_OK;
}

bool dims_ok(int64_t rows, int64_t cols) {
  return rows >= 0 && cols >= 0 && (rows == 0 || cols <= (int64_t)(INT64_MAX / 8) / rows);
}

}  // namespace

extern "C" tsk_status tsk_array_save(const char* path, const void* host, tsk_prec prec,
                                     int64_t rows, int64_t cols) {
  const size_t es = elt_size((int)prec);
  if (!path || es == 0 || !dims_ok(rows, cols) || (!host && rows * cols > 0)) {
    set_thread_error("tsk_array_save: bad arguments");
    return TSK_EINVAL;
  }
  unsigned char hdr[kArrHeader] = {};
  memcpy(hdr, kArrMagic, 8);
  put_u32(hdr + 8, (uint32_t)prec);
  put_u32(hdr + 12, 0);
  put_u64(hdr + 16, (uint64_t)rows);
  put_u64(hdr + 24, (uint64_t)cols);
  const void* parts[1] = {host};
  const size_t counts[1] = {(size_t)(rows * cols)};
  return write_file("tsk_array_save", path, hdr, kArrHeader, parts, counts, 1, es);
}

extern "C" tsk_status tsk_array_load(const char* path, void* host, int64_t capacity,
                                     tsk_prec* prec, int64_t* rows, int64_t* cols) {
  if (!path || !prec || !rows || !cols || capacity < 0) {
    set_thread_error("tsk_array_load: bad arguments");
    return TSK_EINVAL;
  }
  FILE* f = fopen(path, "rb");
  if (!f) {
    set_thread_error("tsk_array_load: cannot open %s", path);
    return TSK_EINVAL;
  }
  unsigned char hdr[kArrHeader] = {};
  tsk_status st = TSK_OK;
  if (fread(hdr, 1, kArrHeader, f) != (size_t)kArrHeader || memcmp(hdr, kArrMagic, 8) != 0) {
    set_thread_error("tsk_array_load: %s is not a tsk array file", path);
    st = TSK_EINVAL;
  }
  const int p = (int)get_u32(hdr + 8);
  const int64_t r = (int64_t)get_u64(hdr + 16), c = (int64_t)get_u64(hdr + 24);
  const size_t es = elt_size(p);
  if (st == TSK_OK && (es == 0 || get_u32(hdr + 12) != 0 || !dims_ok(r, c))) {
    set_thread_error("tsk_array_load: %s has a malformed header", path);
    st = TSK_EINVAL;
  }
  if (st == TSK_OK) {
    *prec = (tsk_prec)p;
    *rows = r;
    *cols = c;
    if (host) {
      if ((uint64_t)capacity < (uint64_t)(r * c) * es) {
        set_thread_error("tsk_array_load: %s needs %lld bytes, capacity %lld", path,
                         (long long)(r * c * (int64_t)es), (long long)capacity);
        st = TSK_EINVAL;
      } else if (!read_elems(f, host, (size_t)(r * c), es)) {
        set_thread_error("tsk_array_load: %s is shorter than its header says", path);
        st = TSK_EINVAL;
      }
    }
  }
  fclose(f);
  return st;
}

extern "C" tsk_status tsk_refine_save(const char* path, tsk_prec prec, int64_t k, int64_t m,
                                      const tsk_refine_opts* opts,
                                      const tsk_refine_state* state, const void* dS_host,
                                      const void* best_host) {
  const size_t es = (prec == TSK_FP64) ? 8 : (prec == TSK_FP32 ? 4 : 0);
  if (!path || es == 0 || k < 1 || m < 1 || !dims_ok(k, m) || !opts || !state || !dS_host ||
      !best_host || state->step < 0 || state->step > opts->steps) {
    set_thread_error("tsk_refine_save: bad arguments");
    return TSK_EINVAL;
  }
  unsigned char hdr[kRefHeader] = {};
  memcpy(hdr, kRefMagic, 8);
  put_u32(hdr + 8, (uint32_t)prec);
  put_u32(hdr + 12, (uint32_t)state->step);
  put_u64(hdr + 16, (uint64_t)k);
  put_u64(hdr + 24, (uint64_t)m);
  put_f64(hdr + 32, state->best_loss);
  put_f64(hdr + 40, opts->lr);
  put_u64(hdr + 48, opts->seed);
  put_u32(hdr + 56, (uint32_t)opts->steps);
  put_u32(hdr + 60, (uint32_t)opts->batch);
  put_u32(hdr + 64, (uint32_t)opts->eval_every);
  put_u32(hdr + 68, opts->order ? 1u : 0u);
  const void* parts[2] = {dS_host, best_host};
  const size_t counts[2] = {(size_t)(k * m), (size_t)(k * m)};
  return write_file("tsk_refine_save", path, hdr, kRefHeader, parts, counts, 2, es);
}

extern "C" tsk_status tsk_refine_load(const char* path, tsk_prec* prec, int64_t* k, int64_t* m,
                                      tsk_refine_opts* opts, int32_t* order_given,
                                      tsk_refine_state* state, void* dS_host, void* best_host,
                                      int64_t capacity) {
  if (!path || !prec || !k || !m || !opts || !state || capacity < 0 ||
      ((dS_host == nullptr) != (best_host == nullptr))) {
    set_thread_error("tsk_refine_load: bad arguments");
    return TSK_EINVAL;
  }
  FILE* f = fopen(path, "rb");
  if (!f) {
    set_thread_error("tsk_refine_load: cannot open %s", path);
    return TSK_EINVAL;
  }
  unsigned char hdr[kRefHeader] = {};
  tsk_status st = TSK_OK;
  if (fread(hdr, 1, kRefHeader, f) != (size_t)kRefHeader || memcmp(hdr, kRefMagic, 8) != 0) {
    set_thread_error("tsk_refine_load: %s is not a tsk refiner checkpoint", path);
    st = TSK_EINVAL;
  }
  const int p = (int)get_u32(hdr + 8);
  const int32_t step = (int32_t)get_u32(hdr + 12);
  const int64_t kk = (int64_t)get_u64(hdr + 16), mm = (int64_t)get_u64(hdr + 24);
  const int32_t steps = (int32_t)get_u32(hdr + 56), batch = (int32_t)get_u32(hdr + 60),
                every = (int32_t)get_u32(hdr + 64);
  const uint32_t og = get_u32(hdr + 68);
  const size_t es = (p == TSK_FP64) ? 8 : (p == TSK_FP32 ? 4 : 0);
  if (st == TSK_OK && (es == 0 || kk < 1 || mm < 1 || !dims_ok(kk, mm) || steps < 0 ||
                       step < 0 || step > steps || batch < 1 || every < 1 || og > 1)) {
    set_thread_error("tsk_refine_load: %s has a malformed header", path);
    st = TSK_EINVAL;
  }
  if (st == TSK_OK) {
    *prec = (tsk_prec)p;
    *k = kk;
    *m = mm;
    tsk_default_refine_options(opts);
    opts->steps = steps;
    opts->batch = batch;
    opts->eval_every = every;
    opts->lr = get_f64(hdr + 40);
    opts->seed = get_u64(hdr + 48);
    opts->order = nullptr;
    if (order_given) *order_given = (int32_t)og;
    state->step = step;
    state->best_loss = get_f64(hdr + 32);
    if (dS_host) {
      const uint64_t need = (uint64_t)(kk * mm) * es;
      if ((uint64_t)capacity < need) {
        set_thread_error("tsk_refine_load: %s needs %llu bytes per array, capacity %lld", path,
                         (unsigned long long)need, (long long)capacity);
        st = TSK_EINVAL;
      } else if (!read_elems(f, dS_host, (size_t)(kk * mm), es) ||
                 !read_elems(f, best_host, (size_t)(kk * mm), es)) {
        set_thread_error("tsk_refine_load: %s is shorter than its header says", path);
        st = TSK_EINVAL;
      }
    }
  }
  fclose(f);
  return st;
}
