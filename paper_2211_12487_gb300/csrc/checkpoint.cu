// Checkpoint file of a TT-ICE decomposition (host code only): the cores are the compressed form of
// the accumulation (Sec. 5.3), so a checkpoint holds the mode sizes, eps, the heuristics, the ranks,
// the cores U_1..U_d and the last core, and nothing else.  The layout is documented in ttice.h.
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "ttice_internal.cuh"

namespace {

constexpr char kMagic[8] = {'T', 'T', 'I', 'C', 'E', 'C', 'K', '1'};
constexpr int32_t kVersion = 1;

// FNV-1a (64-bit) over the bytes written so far
struct Hash {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  }
};

// Values are written in the host's byte order, which the format requires to be little-endian.
bool host_little_endian() {
  const uint32_t one = 1;
  unsigned char b;
  memcpy(&b, &one, 1);
  return b == 1;
}

struct Writer {
  explicit Writer(FILE* file) : f(file) {}
  FILE* f;
  Hash hash;
  bool ok = true;
  void put(const void* p, size_t n) {
    if (!ok || n == 0) return;
    ok = fwrite(p, 1, n, f) == n;
    hash.add(p, n);
  }
  template <typename T>
  void val(T v) { put(&v, sizeof(T)); }
};

struct Reader {
  explicit Reader(FILE* file) : f(file) {}
  FILE* f;
  Hash hash;
  bool ok = true;
  void get(void* p, size_t n) {
    if (!ok || n == 0) return;
    ok = fread(p, 1, n, f) == n;
    if (ok) hash.add(p, n);
  }
  template <typename T>
  T val() {
    T v{};
    get(&v, sizeof(T));
    return v;
  }
};

// Shape checks shared by the writer and the reader: 1 <= d <= 16, positive mode sizes, r_0 = 1,
// 0 <= r_i <= r_{i-1} n_i, n_obs >= 0, and every array size (elements and bytes) representable in
// int64 (checked products: a crafted header cannot make a size wrap around).
bool valid_shape(int d, const int64_t* dims, const int64_t* ranks, int64_t n_obs) {
  if (d < 1 || d > ttice::kMaxD || n_obs < 0 || ranks[0] != 1) return false;
  for (int i = 0; i < d; ++i) {
    int64_t bound = 0;
    if (dims[i] < 1 || ranks[i + 1] < 0 || __builtin_mul_overflow(ranks[i], dims[i], &bound) ||
        ranks[i + 1] > bound)
      return false;
  }
  return ttice::checked_shape_elems(d, dims, ranks, n_obs, nullptr, nullptr, nullptr);
}

}  // namespace

extern "C" {

int ttice_checkpoint_write(const char* path, int d, const int64_t* dims, double eps,
                           const ttice_heuristics* heur, const int64_t* ranks,
                           const double* const* cores, const double* last, int64_t n_obs) {
  if (!path || !dims || !heur || !ranks || !host_little_endian()) return TTICE_EINVAL;
  if (!valid_shape(d, dims, ranks, n_obs) || !(eps > 0.0 && eps < 1.0)) return TTICE_EINVAL;
  int64_t ce[ttice::kMaxD] = {}, le = 0;
  ttice::checked_shape_elems(d, dims, ranks, n_obs, ce, &le, nullptr);  // valid_shape checked it
  for (int i = 0; i < d; ++i)
    if (ce[i] > 0 && (!cores || !cores[i])) return TTICE_EINVAL;
  if (le > 0 && !last) return TTICE_EINVAL;
  FILE* f = fopen(path, "wb");
  if (!f) return TTICE_EINVAL;
  Writer w(f);
  w.put(kMagic, sizeof(kMagic));
  w.val<int32_t>(kVersion);
  w.val<int32_t>(d);
  for (int i = 0; i < d; ++i) w.val<int64_t>(dims[i]);
  w.val<double>(eps);
  w.val<int32_t>(heur->skip_mode);
  w.val<int32_t>(heur->subselect);
  w.val<int32_t>(heur->eps_upd_mode);
  w.val<double>(heur->occupancy_tau);
  w.val<int32_t>(heur->precision);
  w.val<int32_t>(heur->input_dtype);
  for (int i = 0; i <= d; ++i) w.val<int64_t>(ranks[i]);
  w.val<int64_t>(n_obs);
  for (int i = 0; i < d; ++i) w.put(cores[i], (size_t)ce[i] * sizeof(double));
  w.put(last, (size_t)le * sizeof(double));
  const uint64_t sum = w.hash.h;
  if (w.ok) w.ok = fwrite(&sum, 1, sizeof(sum), f) == sizeof(sum);
  const bool closed = fclose(f) == 0;
  return (w.ok && closed) ? TTICE_OK : TTICE_EINVAL;
}

int ttice_checkpoint_read(const char* path, int* d, int64_t* dims, double* eps, ttice_heuristics* heur,
                          int64_t* ranks, int64_t* n_obs, double* const* cores, double* last) {
  if (!path || !d || !dims || !eps || !heur || !ranks || !n_obs || !host_little_endian())
    return TTICE_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return TTICE_EINVAL;
  Reader r(f);
  char magic[8];
  r.get(magic, sizeof(magic));
  const int32_t version = r.val<int32_t>();
  const int32_t dd = r.val<int32_t>();
  int rc = TTICE_OK;
  if (!r.ok || memcmp(magic, kMagic, sizeof(kMagic)) != 0 || version != kVersion || dd < 1 ||
      dd > ttice::kMaxD)
    rc = TTICE_EINVAL;
  int64_t dm[ttice::kMaxD] = {}, rk[ttice::kMaxD + 1] = {};
  ttice_heuristics hh{};
  double e = 0.0;
  int64_t nob = 0;
  if (rc == TTICE_OK) {
    for (int i = 0; i < dd; ++i) dm[i] = r.val<int64_t>();
    e = r.val<double>();
    hh.skip_mode = r.val<int32_t>();
    hh.subselect = r.val<int32_t>();
    hh.eps_upd_mode = r.val<int32_t>();
    hh.occupancy_tau = r.val<double>();
    hh.precision = r.val<int32_t>();
    hh.input_dtype = r.val<int32_t>();
    for (int i = 0; i <= dd; ++i) rk[i] = r.val<int64_t>();
    nob = r.val<int64_t>();
    if (!r.ok || !valid_shape(dd, dm, rk, nob) || !(e > 0.0 && e < 1.0)) rc = TTICE_EINVAL;
  }
  // the file must be exactly as long as its header says, checked before anything is sized from it
  // (valid_shape has checked that the element counts and their byte count fit in int64)
  int64_t ce[ttice::kMaxD] = {}, le = 0;
  if (rc == TTICE_OK) {
    int64_t elems = 0;
    ttice::checked_shape_elems(dd, dm, rk, nob, ce, &le, &elems);
    const int64_t header = 8 + 4 + 4 + 8 * (int64_t)dd + 8 + 3 * 4 + 8 + 2 * 4 + 8 * (int64_t)(dd + 1) + 8;
    const int64_t total = header + 8 * elems + 8;  // < INT64_MAX: elems <= INT64_MAX / 8 - 1 by then
    const long pos = ftell(f);
    long size = -1;
    if (pos >= 0 && fseek(f, 0, SEEK_END) == 0) size = ftell(f);
    if (size < 0 || fseek(f, pos, SEEK_SET) != 0 || total != (int64_t)size) rc = TTICE_EINVAL;
  }
  if (rc == TTICE_OK) {
    *d = dd;
    for (int i = 0; i < dd; ++i) dims[i] = dm[i];
    *eps = e;
    *heur = hh;
    for (int i = 0; i <= dd; ++i) ranks[i] = rk[i];
    *n_obs = nob;
  }
  // first call (no buffers): the header only
  if (rc != TTICE_OK || !cores) {
    fclose(f);
    return rc;
  }
  for (int i = 0; i < dd && rc == TTICE_OK; ++i) {
    const size_t n = (size_t)ce[i];
    if (n > 0 && !cores[i]) rc = TTICE_EINVAL;
    else r.get(cores[i], n * sizeof(double));
  }
  const size_t nl = (size_t)le;
  if (rc == TTICE_OK) {
    if (nl > 0 && !last) rc = TTICE_EINVAL;
    else r.get(last, nl * sizeof(double));
  }
  if (rc == TTICE_OK) {
    const uint64_t expect = r.hash.h;
    uint64_t sum = 0;
    const bool got = fread(&sum, 1, sizeof(sum), f) == sizeof(sum);
    char extra;
    const bool at_end = fread(&extra, 1, 1, f) == 0;
    if (!r.ok || !got || sum != expect || !at_end) rc = TTICE_EINVAL;
  }
  fclose(f);
  return rc;
}

}  // extern "C"
