// pt_host.cpp -- host side of libpt: argument checks, the integer energy scale, the FP64
// threshold tables (built once per problem on the host), device allocation and the C ABI of
// include/pt.h. All compute happens in the kernels; nothing here falls back to the CPU.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <atomic>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "pt.h"
#include "pt_batch.h"
#include "pt_debug.cuh"
#include "pt_internal.h"
#include "pt_launch.h"
#include "pt_flip.h"
#include "pt_persist.h"

using namespace ptb;

namespace {
thread_local std::string g_last_error;
}  // namespace

int ptb::fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

namespace {

struct Allocator {
  pt_alloc_fn alloc = nullptr;
  pt_free_fn free = nullptr;
  void* ctx = nullptr;
};
std::mutex g_mu;
Allocator g_alloc;

constexpr uint64_t kTwo32 = 1ull << 32;

}  // namespace

namespace ptb {
BatchTuning batch_tuning() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_batch_tuning;
}
}  // namespace ptb

namespace {

// ---------------------------------------------------------------------------------------
// Exact integer energies (the quantisation of include/pt.h)
// ---------------------------------------------------------------------------------------
int quantise(double J, double h, int64_t* s_out, int64_t* Ji, int64_t* hi) {
  if (!std::isfinite(J) || !std::isfinite(h)) return PT_EINVAL;
  for (int64_t s = 1; s <= 1000; ++s) {
    const double a = (double)s * J, b = (double)s * h;
    const double ra = std::nearbyint(a), rb = std::nearbyint(b);
    if (std::fabs(a - ra) <= 1e-9 && std::fabs(b - rb) <= 1e-9) {
      if (std::fabs(ra) > 1048576.0 || std::fabs(rb) > 1048576.0) return PT_EINVAL;
      *s_out = s;
      *Ji = (int64_t)ra;
      *hi = (int64_t)rb;
      return PT_OK;
    }
  }
  return PT_EINVAL;
}

// Metropolis threshold of Eq. 1 (Boltzmann ratio of Eq. 2) as a 33-bit integer.
uint64_t spin_threshold(double beta, int64_t dE_int, int64_t s) {
  if (dE_int <= 0) return kTwo32;
  const double x = (beta * (double)dE_int) / (double)s;
  return (uint64_t)std::floor(4294967296.0 * std::exp(-x));
}

// Swap threshold of Sec. 3: the paper's Barker form 1 / (1 + e^y) with the +-44 cut-offs,
// or (option) the Metropolis form min(1, e^-y), y = (beta_hi - beta_lo) n / s.
uint64_t swap_rule(double beta_lo, double beta_hi, int64_t n, int64_t s, int rule) {
  const double y = ((beta_hi - beta_lo) * (double)n) / (double)s;
  if (rule == PT_SWAP_METROPOLIS) {
    if (y <= 0.0) return kTwo32;
    if (y > 44.0) return 0;
    return (uint64_t)std::floor(4294967296.0 * std::exp(-y));
  }
  if (y > 44.0) return 0;
  if (y < -44.0) return kTwo32;
  return (uint64_t)std::floor(4294967296.0 / (1.0 + std::exp(y)));
}

// The exchange threshold of one temperature pair as a function of n: constant below n_lo
// and above n_hi, tabulated in between at the n that are multiples of 2^shift (table_shift:
// no other n can occur). S(n) is monotone in n (y is linear in n and both
// forms are monotone in y), so the saturated ranges are found by bisection and then checked
// at their edges. With reach > 0 only |n| <= reach can occur (a lattice's largest energy
// difference): the table then covers the non-saturated n within [-reach, reach] only, and
// when that is all of [-reach, reach] it is tabulated whole, without a search; a lookup of
// any |n| <= reach gives S(n) either way.
struct PairTable {
  int64_t n_lo = 1, n_hi = 0;
  uint64_t S_below = 0, S_above = 0;
  std::vector<uint32_t> vals;
};

// The largest multiple of step <= x, and the smallest >= x (step > 0).
int64_t floor_multiple(int64_t x, int64_t step) {
  const int64_t q = x / step;
  return (q * step > x ? q - 1 : q) * step;
}
int64_t ceil_multiple(int64_t x, int64_t step) { return -floor_multiple(-x, step); }

// Every energy difference n = E_int(a) - E_int(b) is a multiple of gcd(4 J_int, 2 h_int):
// flipping one spin changes the number of unsatisfied bonds by 4 - 2 k (even), so the bond
// sum of Eq. 3 moves in steps of 4 from its all-up value 2 L^2, and the magnetisation in
// steps of 2 from L^2. The exchange tables keep only the n that are multiples of the power
// of two in that gcd (4 for J = 1, h = 0): a quarter of the entries.
int table_shift(int64_t Ji, int64_t hi) {
  uint64_t a = 4 * (uint64_t)(Ji < 0 ? -Ji : Ji), b = 2 * (uint64_t)(hi < 0 ? -hi : hi);
  while (b) {
    const uint64_t r = a % b;
    a = b;
    b = r;
  }
  if (a == 0) return 0;
  int k = 0;
  while (!(a & 1)) {
    a >>= 1;
    ++k;
  }
  return k;
}

// Tabulates S at n_lo, n_lo + 2^shift, ..., n_hi, after rounding n_lo up and n_hi down to
// multiples of 2^shift (no multiple lies in the parts cut off, so lookups of multiples
// below or above the new range still get S_below / S_above).
int fill_pair_table(double blo, double bhi, int64_t s, int rule, int shift, PairTable* t) {
  const double d = bhi - blo;
  const int64_t step = (int64_t)1 << shift;
  t->n_lo = ceil_multiple(t->n_lo, step);
  t->n_hi = floor_multiple(t->n_hi, step);
  const int64_t len = t->n_hi >= t->n_lo ? (t->n_hi - t->n_lo) / step + 1 : 0;
  t->vals.resize((size_t)len);
  uint64_t prev = swap_rule(blo, bhi, t->n_lo - step, s, rule);
  for (int64_t j = 0; j < len; ++j) {
    const int64_t n = t->n_lo + j * step;
    const uint64_t v = swap_rule(blo, bhi, n, s, rule);
    if (v >= kTwo32) return fail(PT_EINTERNAL, "exchange table entry saturates inside");
    if ((d > 0 && v > prev) || (d < 0 && v < prev))
      return fail(PT_EINTERNAL, "exchange threshold not monotone at n = %lld", (long long)n);
    prev = v;
    t->vals[(size_t)j] = (uint32_t)v;
  }
  return PT_OK;
}

int build_pair_table(double blo, double bhi, int64_t s, int rule, int64_t reach, int shift,
                     PairTable* out) {
  PairTable t;
  const double d = bhi - blo;
  if (d == 0.0) {  // y = 0 for every n
    t.S_below = t.S_above = swap_rule(blo, bhi, 0, s, rule);
    *out = std::move(t);
    return PT_OK;
  }
  // beyond +-N the cut-offs decide (|y| > 44)
  const double nmax = std::ceil(45.0 * (double)s / std::fabs(d)) + 2.0;
  if (reach > 0 && (double)reach + 2.0 < nmax) {
    // every reachable n lies inside the search range: tabulate [-reach, reach] whole
    t.n_lo = -reach;
    t.n_hi = reach;
    t.S_below = swap_rule(blo, bhi, -reach - 1, s, rule);
    t.S_above = swap_rule(blo, bhi, reach + 1, s, rule);
    if (t.S_below >= kTwo32 || t.S_above >= kTwo32 || t.S_below == 0 || t.S_above == 0) {
      // a saturated end inside [-reach - 1, reach + 1]: search for the edges instead
    } else {
      const int rc = fill_pair_table(blo, bhi, s, rule, shift, &t);
      if (rc) return rc;
      *out = std::move(t);
      return PT_OK;
    }
  }
  if (nmax > 4.0e9) return fail(PT_EINVAL, "temperature pair too close: |dbeta| = %g", d);
  const int64_t N = (int64_t)nmax;
  t.S_below = swap_rule(blo, bhi, -N, s, rule);
  t.S_above = swap_rule(blo, bhi, N, s, rule);
  // n_lo = smallest n with S(n) != S_below
  int64_t lo = -N, hi = N;  // S(lo) == S_below, search in (lo, hi]
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (swap_rule(blo, bhi, mid, s, rule) != t.S_below) hi = mid; else lo = mid;
  }
  t.n_lo = hi;
  lo = -N;
  hi = N;  // largest n with S(n) != S_above: S(hi) == S_above, search in [lo, hi)
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (swap_rule(blo, bhi, mid, s, rule) != t.S_above) lo = mid; else hi = mid;
  }
  t.n_hi = lo;
  if (t.n_hi < t.n_lo) return fail(PT_EINTERNAL, "empty exchange table");
  if (swap_rule(blo, bhi, t.n_lo - 1, s, rule) != t.S_below ||
      swap_rule(blo, bhi, t.n_hi + 1, s, rule) != t.S_above)
    return fail(PT_EINTERNAL, "exchange table edges inconsistent");
  if (reach > 0) {
    // keep the reachable part; an empty one still sends every |n| <= reach to the right
    // constant
    const int64_t lo_r = std::max(t.n_lo, -reach), hi_r = std::min(t.n_hi, reach);
    if (lo_r <= hi_r) {
      t.n_lo = lo_r;
      t.n_hi = hi_r;
    } else if (t.n_lo > reach) {  // every reachable n is below the table
      t.n_lo = reach + 1;
      t.n_hi = reach;
    } else {  // every reachable n is above it
      t.n_lo = -reach;
      t.n_hi = -reach - 1;
    }
  }
  const int rc = fill_pair_table(blo, bhi, s, rule, shift, &t);
  if (rc) return rc;
  *out = std::move(t);
  return PT_OK;
}

// Tables depend only on (beta_lo, beta_hi, s, rule, reach, shift); requests with the same
// ladder, lattice reach and stride share them.
struct PairKey {
  uint64_t blo, bhi;
  int64_t s;
  int rule;
  int64_t reach;
  int shift;
  bool operator<(const PairKey& o) const {
    return std::tie(blo, bhi, s, rule, reach, shift) <
           std::tie(o.blo, o.bhi, o.s, o.rule, o.reach, o.shift);
  }
};
std::mutex g_table_mu;
std::map<PairKey, std::shared_ptr<const PairTable>> g_tables;
size_t g_table_bytes = 0;
constexpr size_t kTableCacheCap = size_t(2) << 30;

// The largest |n| = |E_int(a) - E_int(b)| on an L x L lattice: |E_int| <= 2 L^2 |J_int| +
// L^2 |h_int| (2 L^2 bonds, L^2 spins).
int64_t energy_reach(int L, int64_t Ji, int64_t hi) {
  const int64_t L2 = (int64_t)L * L;
  return 2 * (2 * L2 * (Ji < 0 ? -Ji : Ji) + L2 * (hi < 0 ? -hi : hi));
}

// reach: the largest |n| that can occur (0: any n). The reach shapes the table only when
// it is inside the pair's saturation range (a small lattice on a dense ladder); otherwise
// the whole table is built and shared by every lattice size, so problems that differ only
// in L share it.
bool reach_shapes(double blo, double bhi, int64_t s, int64_t reach) {
  const double d = std::fabs(bhi - blo);
  const double nmax = d == 0.0 ? 0.0 : std::ceil(45.0 * (double)s / d) + 2.0;
  return reach > 0 && (double)reach + 2.0 < nmax;
}

int get_pair_table(double blo, double bhi, int64_t s, int rule, int64_t reach, int shift,
                   std::shared_ptr<const PairTable>* out) {
  if (!reach_shapes(blo, bhi, s, reach)) reach = 0;
  PairKey key;
  memcpy(&key.blo, &blo, 8);
  memcpy(&key.bhi, &bhi, 8);
  key.s = s;
  key.rule = rule;
  key.reach = reach;
  key.shift = shift;
  {
    std::lock_guard<std::mutex> lk(g_table_mu);
    auto it = g_tables.find(key);
    if (it != g_tables.end()) {
      *out = it->second;
      return PT_OK;
    }
  }
  auto t = std::make_shared<PairTable>();
  const int rc = build_pair_table(blo, bhi, s, rule, reach, shift, t.get());
  if (rc != PT_OK) return rc;
  std::lock_guard<std::mutex> lk(g_table_mu);
  if (g_table_bytes > kTableCacheCap) {
    g_tables.clear();
    g_table_bytes = 0;
  }
  g_table_bytes += t->vals.size() * 4;
  g_tables[key] = t;
  *out = t;
  return PT_OK;
}

// The tables of a ladder's R - 1 adjacent pairs; long ladders are built on up to 16 host
// threads (the tables are independent and the cache is shared). An error in any of them is
// reported on the calling thread.
int get_ladder_tables(const double* betas, int R, int64_t s, int rule, int64_t reach,
                      int shift, std::vector<std::shared_ptr<const PairTable>>* out) {
  const int npairs = std::max(R - 1, 0);
  out->assign((size_t)npairs, nullptr);
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nthreads = npairs < 64 ? 1 : std::min(std::min(hw, 16), npairs / 32);
  std::atomic<int> next{0};
  std::vector<int> rcs((size_t)nthreads, PT_OK);
  std::vector<std::string> msgs((size_t)nthreads);
  auto work = [&](int w) {
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= npairs) return;
      const int rc =
          get_pair_table(betas[k], betas[k + 1], s, rule, reach, shift, &(*out)[(size_t)k]);
      if (rc) {
        rcs[(size_t)w] = rc;
        msgs[(size_t)w] = g_last_error;
        return;
      }
    }
  };
  if (nthreads == 1) {
    work(0);
  } else {
    std::vector<std::thread> pool;
    for (int w = 0; w < nthreads; ++w) pool.emplace_back(work, w);
    for (std::thread& th : pool) th.join();
  }
  for (int w = 0; w < nthreads; ++w)
    if (rcs[(size_t)w]) return fail(rcs[(size_t)w], "%s", msgs[(size_t)w].c_str());
  return PT_OK;
}

// ---------------------------------------------------------------------------------------
// Device
// ---------------------------------------------------------------------------------------
int current_device(DeviceInfo* info) {
  static std::mutex mu;
  static std::map<int, DeviceInfo> cache;
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return fail(PT_ENODEV, "no CUDA device: %s", cudaGetErrorString(err));
  }
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it == cache.end()) {
    cudaDeviceProp prop;
    err = cudaGetDeviceProperties(&prop, dev);
    if (err != cudaSuccess) return fail(PT_ENODEV, "%s", cudaGetErrorString(err));
    if (!(prop.major == 10 && prop.minor == 3))
      return fail(PT_ENODEV, "device %d is sm_%d%d; libpt is built for sm_103a only", dev,
                  prop.major, prop.minor);
    DeviceInfo d;
    d.device = dev;
    d.sms = prop.multiProcessorCount;
    d.cc_major = prop.major;
    d.cc_minor = prop.minor;
    d.smem_optin = prop.sharedMemPerBlockOptin;
    it = cache.emplace(dev, d).first;
  }
  *info = it->second;
  return PT_OK;
}

// Sub-buffer layout of the single device allocation of a problem.
struct Layout {
  size_t spins, T_temp, planes, temp_of_slot, slot_of_temp, cnt, E_slot, M_slot, attempted,
      accepted, pairs, table, status, total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(int L, int R, int W, int mode, size_t table_entries) {
  Layout l;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t npairs = (size_t)std::max(R - 1, 1);
  l.spins = take((size_t)W * L * L * 4);
  l.T_temp = take((size_t)R * kClasses * 8);
  l.planes = take((size_t)W * (mode == kModeFerro ? sizeof(PlaneFerro) : sizeof(PlaneGeneric)));
  l.temp_of_slot = take((size_t)R * 4);
  l.slot_of_temp = take((size_t)R * 4);
  l.cnt = take(count_words(W) * 4);
  l.E_slot = take((size_t)R * 8);
  l.M_slot = take((size_t)R * 8);
  l.attempted = take(npairs * 8);
  l.accepted = take(npairs * 8);
  l.pairs = take(npairs * sizeof(SwapPair));
  l.table = take(std::max<size_t>(table_entries, 1) * 4);
  l.status = take(64);
  l.total = off;
  return l;
}

int check_args(int L, const double* betas, int R, double J, double h, int64_t* s, int64_t* Ji,
               int64_t* hi) {
  if (L < 4 || L > PT_MAX_L || (L & 1))
    return fail(PT_EINVAL, "L = %d must be even and within [4, %d]", L, PT_MAX_L);
  if (R < 1 || R > PT_MAX_R) return fail(PT_EINVAL, "R = %d outside [1, %d]", R, PT_MAX_R);
  if (!betas) return fail(PT_EINVAL, "betas is NULL");
  for (int k = 0; k < R; ++k)
    if (!std::isfinite(betas[k]) || betas[k] < 0.0)
      return fail(PT_EINVAL, "betas[%d] = %g must be finite and >= 0", k, betas[k]);
  if (quantise(J, h, s, Ji, hi) != PT_OK)
    return fail(PT_EINVAL, "J = %g, h = %g have no common integer scale s <= 1000 (or exceed "
                "2^20 after scaling)", J, h);
  return PT_OK;
}

int mode_for(int64_t J_int, int64_t h_int) {
  return (h_int == 0 && J_int > 0) ? kModeFerro : kModeGeneric;
}

// ---------------------------------------------------------------------------------------
// Creation images. A problem's allocation from its thresholds to its end (thresholds by
// temperature, identity maps, zeroed planes, counts, energies and counters, pair
// descriptors, exchange tables) is a function of the ladder, the quantised couplings, the
// swap rule and the lattice reach where it shapes a table; the seed only drives the initial
// spins, which are drawn on the device. Its offsets from the thresholds do not depend on L.
// Images up to kImageMaxBytes are built once into page-locked host memory and kept (up to
// g_image_limit in all, pt_set_image_cache_limit), so a creation queues one asynchronous
// copy and does no table
// work on the host. Larger ones (long ladders on large lattices) are built per creation in
// pageable memory. A problem holds its page-locked image until pt_destroy has synchronised
// its stream, so dropping images from the cache never frees one that a copy still reads.
// ---------------------------------------------------------------------------------------
struct ImageKey {
  std::vector<uint64_t> betas;  // bit patterns
  int64_t s, Ji, hi, reach;     // reach: 0 unless it shapes one of the tables
  int rule;
  bool operator<(const ImageKey& o) const {
    return std::tie(s, Ji, hi, reach, rule, betas) <
           std::tie(o.s, o.Ji, o.hi, o.reach, o.rule, o.betas);
  }
};

struct Image {
  std::vector<uint8_t> pageable;  // the bytes, unless page-locked
  uint8_t* locked = nullptr;      // cudaHostAlloc'd bytes
  size_t bytes = 0;
  size_t entries = 0;             // exchange table entries (for the layout)
  const uint8_t* data() const { return locked ? locked : pageable.data(); }
  Image() = default;
  Image(const Image&) = delete;
  Image& operator=(const Image&) = delete;
  ~Image() {
    if (locked) cudaFreeHost(locked);
  }
};

std::mutex g_image_mu;
std::map<ImageKey, std::shared_ptr<const Image>> g_images;
size_t g_image_bytes = 0;
constexpr size_t kImageMaxBytes = size_t(64) << 20;
size_t g_image_limit = size_t(1) << 30;

// Builds the image of a problem with this ladder and layout parameters.
// The bytes go to page-locked memory when they are at most lock_max.
int build_image(int L, const double* betas, int R, int64_t s, int64_t Ji, int64_t hi, int rule,
                int64_t reach, int shift, int mode, size_t lock_max,
                std::shared_ptr<Image>* out) {
  // thresholds by temperature, class c = 2 k + (sigma == +1)
  std::vector<uint64_t> T_temp((size_t)R * kClasses);
  for (int k = 0; k < R; ++k)
    for (int kk = 0; kk <= 4; ++kk)
      for (int up = 0; up <= 1; ++up) {
        const int64_t sigma = up ? 1 : -1;
        const int64_t nb = 4 - 2 * kk;  // sigma * sum of neighbour spins
        const int64_t dE = 2 * (Ji * nb - hi * sigma);
        T_temp[(size_t)k * kClasses + 2 * kk + up] = spin_threshold(betas[k], dE, s);
      }
  if (mode == kModeFerro)
    for (int k = 0; k < R; ++k)
      if (T_temp[(size_t)k * kClasses + 1] > T_temp[(size_t)k * kClasses + 3])
        return fail(PT_EINTERNAL, "threshold order violated at temperature %d", k);

  // exchange tables
  const int npairs = std::max(R - 1, 1);
  std::vector<std::shared_ptr<const PairTable>> tabs;
  std::vector<SwapPair> pairs((size_t)npairs);
  size_t entries = 0;
  int rc = get_ladder_tables(betas, R, s, rule, reach, shift, &tabs);
  if (rc) return rc;
  for (int k = 0; k + 1 < R; ++k) {
    const std::shared_ptr<const PairTable>& t = tabs[(size_t)k];
    pairs[k].n_lo = t->n_lo;
    pairs[k].n_hi = t->n_hi;
    pairs[k].S_below = t->S_below;
    pairs[k].S_above = t->S_above;
    pairs[k].offset = (int64_t)entries;
    entries += t->vals.size();
  }

  const int W = (R + 31) / 32;
  const Layout lay = make_layout(L, R, W, mode, entries);
  auto img = std::make_shared<Image>();
  img->bytes = lay.total - lay.T_temp;
  img->entries = entries;
  uint8_t* dst = nullptr;
  if (img->bytes <= lock_max &&
      cudaHostAlloc((void**)&img->locked, img->bytes, cudaHostAllocPortable) == cudaSuccess) {
    dst = img->locked;
    memset(dst, 0, img->bytes);
  } else {
    cudaGetLastError();
    img->locked = nullptr;
    img->pageable.assign(img->bytes, 0);
    dst = img->pageable.data();
  }
  auto put = [&](size_t off, const void* src, size_t bytes) {
    memcpy(dst + (off - lay.T_temp), src, bytes);
  };
  put(lay.T_temp, T_temp.data(), T_temp.size() * 8);
  std::vector<int32_t> ident(R);
  for (int r = 0; r < R; ++r) ident[r] = r;
  put(lay.temp_of_slot, ident.data(), R * 4);
  put(lay.slot_of_temp, ident.data(), R * 4);
  put(lay.pairs, pairs.data(), pairs.size() * sizeof(SwapPair));
  for (int k = 0; k + 1 < R; ++k)
    if (!tabs[k]->vals.empty())
      put(lay.table + (size_t)pairs[k].offset * 4, tabs[k]->vals.data(), tabs[k]->vals.size() * 4);
  *out = std::move(img);
  return PT_OK;
}

// The creation image of a problem: from the cache, or built (and cached when it could be
// page-locked).
int get_image(int L, const double* betas, int R, int64_t s, int64_t Ji, int64_t hi, int rule,
              int mode, std::shared_ptr<const Image>* out) {
  int64_t reach = energy_reach(L, Ji, hi);
  bool shapes = false;
  for (int k = 0; k + 1 < R && !shapes; ++k) shapes = reach_shapes(betas[k], betas[k + 1], s, reach);
  if (!shapes) reach = 0;
  ImageKey key;
  key.betas.resize((size_t)R);
  memcpy(key.betas.data(), betas, (size_t)R * 8);
  key.s = s;
  key.Ji = Ji;
  key.hi = hi;
  key.reach = reach;
  key.rule = rule;
  {
    std::lock_guard<std::mutex> lk(g_image_mu);
    auto it = g_images.find(key);
    if (it != g_images.end()) {
      *out = it->second;
      return PT_OK;
    }
  }
  size_t lock_max;
  {
    std::lock_guard<std::mutex> lk(g_image_mu);
    lock_max = std::min(kImageMaxBytes, g_image_limit);
  }
  std::shared_ptr<Image> img;
  const int rc = build_image(L, betas, R, s, Ji, hi, rule, reach, table_shift(Ji, hi), mode,
                             lock_max, &img);
  if (rc) return rc;
  if (img->locked) {
    std::lock_guard<std::mutex> lk(g_image_mu);
    if (g_image_bytes + img->bytes > g_image_limit) {
      g_images.clear();  // images still held by problems stay alive until their destroy
      g_image_bytes = 0;
    }
    auto ins = g_images.emplace(std::move(key), img);
    if (ins.second) g_image_bytes += img->bytes;
  }
  *out = std::move(img);
  return PT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Problem object
// ---------------------------------------------------------------------------------------
namespace ptb {

int problem_fail(pt_problem* p, int code, const char* what, cudaError_t err) {
  p->poisoned = code;
  return fail(code, "%s: %s", what, cudaGetErrorString(err));
}

int problem_check(pt_problem* p) {
  if (!p) return fail(PT_EINVAL, "problem is NULL");
  if (p->poisoned) return fail(PT_ESTATE, "problem poisoned by an earlier failure (%s)",
                                pt_strerror(p->poisoned));
  return PT_OK;
}

int problem_device_guard(pt_problem* p) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return fail(PT_ENODEV, "cudaGetDevice failed");
  if (cur != p->dev_info.device) {
    const cudaError_t err = cudaSetDevice(p->dev_info.device);
    if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "cudaSetDevice", err);
  }
  return PT_OK;
}

}  // namespace ptb

namespace {

void* dev_alloc(size_t bytes, cudaStream_t st, Allocator* used) {
  std::lock_guard<std::mutex> lk(g_mu);
  *used = g_alloc;
  if (g_alloc.alloc) return g_alloc.alloc(bytes, (void*)st, g_alloc.ctx);
  void* ptr = nullptr;
  if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return ptr;
}

void dev_free(void* ptr, cudaStream_t st, const Allocator& a) {
  if (!ptr) return;
  if (a.free)
    a.free(ptr, (void*)st, a.ctx);
  else
    cudaFree(ptr);
}

// Host copy of one plane (both colours) of the problem.
int read_plane(pt_problem* p, int w, std::vector<uint32_t>* buf) {
  buf->resize((size_t)p->L * p->L);
  cudaError_t err = cudaMemcpyAsync(buf->data(), p->dev.spins + (size_t)w * p->L * p->L,
                                    buf->size() * 4, cudaMemcpyDeviceToHost, p->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "reading spins", err);
  return PT_OK;
}

int slot_at_temperature(pt_problem* p, int k, int* slot) {
  int32_t r = -1;
  cudaError_t err = cudaMemcpyAsync(&r, p->dev.slot_of_temp + k, 4, cudaMemcpyDeviceToHost,
                                    p->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "reading slot map", err);
  if (r < 0 || r >= p->R) return fail(PT_EINTERNAL, "slot map corrupt");
  *slot = r;
  return PT_OK;
}

// Energy pass + finalize so that E_slot / M_slot describe the current state.
int refresh_observables(pt_problem* p) {
  cudaError_t err = launch_energy(p->dev, p->dev_info, p->stream);
  if (err == cudaSuccess) err = launch_exchange(p->dev, p->e, kStepEnergy, p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "energy launch", err);
  return PT_OK;
}

int read_observables(pt_problem* p, std::vector<int64_t>* E, std::vector<int64_t>* M,
                     std::vector<int32_t>* slot_of_temp) {
  int rc = refresh_observables(p);
  if (rc) return rc;
  E->resize(p->R);
  M->resize(p->R);
  slot_of_temp->resize(p->R);
  cudaError_t err = cudaMemcpyAsync(E->data(), p->dev.E_slot, p->R * 8, cudaMemcpyDeviceToHost,
                                    p->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(M->data(), p->dev.M_slot, p->R * 8, cudaMemcpyDeviceToHost, p->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(slot_of_temp->data(), p->dev.slot_of_temp, p->R * 4,
                          cudaMemcpyDeviceToHost, p->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "reading observables", err);
  return PT_OK;
}

}  // namespace

// =======================================================================================
// C ABI
// =======================================================================================
// ---------------------------------------------------------------------------------------
// Checkpoints (include/pt.h documents the byte layout)
// ---------------------------------------------------------------------------------------
namespace {

constexpr char kCkptMagic[8] = {'P', 'T', 'C', 'K', 'P', 'T', '0', '2'};
constexpr size_t kCkptHeader = 72;

size_t ckpt_bytes(int L, int R) {
  const int W = (R + 31) / 32;
  const size_t pairs = (size_t)std::max(R - 1, 0);
  return kCkptHeader + (size_t)R * 8 + (size_t)R * 4 + pairs * 16 + (size_t)W * L * L * 4 + 8;
}

// FNV-1a, 64 bit (Fowler, Noll, Vo)
uint64_t fnv1a64(const uint8_t* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct Writer {
  uint8_t* p;
  template <class T>
  void put(const T& v) {
    memcpy(p, &v, sizeof(T));
    p += sizeof(T);
  }
  void put_bytes(const void* src, size_t n) {
    memcpy(p, src, n);
    p += n;
  }
};

struct Reader {
  const uint8_t* p;
  template <class T>
  T get() {
    T v;
    memcpy(&v, p, sizeof(T));
    p += sizeof(T);
    return v;
  }
};

}  // namespace

extern "C" {

const char* pt_version(void) { return "libpt 0.1 (sm_103a)"; }

const char* pt_strerror(int code) {
  switch (code) {
    case PT_OK: return "ok";
    case PT_EINVAL: return "invalid argument";
    case PT_ENOMEM: return "out of memory";
    case PT_ECUDA: return "CUDA error";
    case PT_ETIMEOUT: return "device wait timed out";
    case PT_ESTATE: return "problem poisoned by an earlier failure";
    case PT_ENODEV: return "no usable sm_103 device";
    case PT_EINTERNAL: return "internal error";
    default: return "unknown error";
  }
}

const char* pt_last_error(void) { return g_last_error.c_str(); }

int pt_quantise(double J, double h, int64_t* s, int64_t* J_int, int64_t* h_int) {
  if (!s || !J_int || !h_int) return fail(PT_EINVAL, "NULL output");
  const int rc = quantise(J, h, s, J_int, h_int);
  if (rc) return fail(rc, "J = %g, h = %g cannot be quantised", J, h);
  return PT_OK;
}

uint64_t pt_spin_threshold(double beta, int64_t dE_int, int64_t s) {
  return spin_threshold(beta, dE_int, s);
}

uint64_t pt_swap_threshold_ex(double beta_lo, double beta_hi, int64_t n, int64_t s, int rule) {
  if (rule != PT_SWAP_BARKER && rule != PT_SWAP_METROPOLIS) return ~uint64_t(0);
  std::shared_ptr<const PairTable> t;
  if (get_pair_table(beta_lo, beta_hi, s, rule, 0, 0, &t) != PT_OK) return ~uint64_t(0);
  if (n < t->n_lo) return t->S_below;
  if (n > t->n_hi) return t->S_above;
  return t->vals[(size_t)(n - t->n_lo)];
}

uint64_t pt_swap_threshold(double beta_lo, double beta_hi, int64_t n, int64_t s) {
  return pt_swap_threshold_ex(beta_lo, beta_hi, n, s, PT_SWAP_BARKER);
}

int pt_set_allocator(pt_alloc_fn alloc, pt_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(PT_EINVAL, "alloc and free must both be set or both be NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  g_alloc.alloc = alloc;
  g_alloc.free = free_fn;
  g_alloc.ctx = ctx;
  return PT_OK;
}

size_t pt_estimate_device_bytes(int L, const double* betas, int R, double J, double h) {
  int64_t s, Ji, hi;
  if (check_args(L, betas, R, J, h, &s, &Ji, &hi) != PT_OK) return 0;
  size_t entries = 0;
  std::vector<std::shared_ptr<const PairTable>> tabs;
  if (get_ladder_tables(betas, R, s, PT_SWAP_BARKER, energy_reach(L, Ji, hi),
                        table_shift(Ji, hi), &tabs) != PT_OK)
    return 0;
  for (const auto& t : tabs) entries += t->vals.size();
  const int W = (R + 31) / 32;
  return make_layout(L, R, W, mode_for(Ji, hi), entries).total;
}

int pt_set_image_cache_limit(size_t bytes) {
  std::lock_guard<std::mutex> lk(g_image_mu);
  g_image_limit = bytes;
  if (g_image_bytes > g_image_limit) {
    g_images.clear();  // images still held by problems stay alive until their destroy
    g_image_bytes = 0;
  }
  return PT_OK;
}

size_t pt_image_cache_bytes(void) {
  std::lock_guard<std::mutex> lk(g_image_mu);
  return g_image_bytes;
}

int pt_create(int L, const double* betas, int R, double J, double h, uint64_t seed,
              pt_problem** out) {
  return pt_create_ex(L, betas, R, J, h, seed, nullptr, out);
}

int pt_create_ex(int L, const double* betas, int R, double J, double h, uint64_t seed,
                 const pt_options* opt, pt_problem** out) {
  if (!out) return fail(PT_EINVAL, "out is NULL");
  *out = nullptr;
  int swap_rule_opt = PT_SWAP_BARKER;
  cudaStream_t stream = 0;
  if (opt) {
    if (opt->size < sizeof(uint32_t) || opt->size > 4096)
      return fail(PT_EINVAL, "pt_options.size = %u", opt->size);
    if (opt->size >= offsetof(pt_options, swap_rule) + sizeof(int32_t))
      swap_rule_opt = opt->swap_rule;
    if (swap_rule_opt != PT_SWAP_BARKER && swap_rule_opt != PT_SWAP_METROPOLIS)
      return fail(PT_EINVAL, "unknown swap rule %d", swap_rule_opt);
    if (opt->size >= offsetof(pt_options, stream) + sizeof(void*))
      stream = (cudaStream_t)opt->stream;
  }
  int64_t s, Ji, hi;
  int rc = check_args(L, betas, R, J, h, &s, &Ji, &hi);
  if (rc) return rc;
  DeviceInfo dev;
  rc = current_device(&dev);
  if (rc) return rc;

  std::unique_ptr<pt_problem> p(new pt_problem());
  p->L = L;
  p->R = R;
  p->W = (R + 31) / 32;
  p->mode = mode_for(Ji, hi);
  p->betas.assign(betas, betas + R);
  p->J = J;
  p->h = h;
  p->s = s;
  p->J_int = Ji;
  p->h_int = hi;
  p->seed = seed;
  p->swap_rule = swap_rule_opt;
  p->dev_info = dev;
  p->stream = stream;

  // thresholds, maps, zeroed buffers, pair descriptors and exchange tables: one image
  std::shared_ptr<const Image> img;
  rc = get_image(L, betas, R, s, Ji, hi, swap_rule_opt, p->mode, &img);
  if (rc) return rc;

  // device memory: one allocation
  const Layout lay = make_layout(L, R, p->W, p->mode, img->entries);
  if (lay.total - lay.T_temp != img->bytes) return fail(PT_EINTERNAL, "creation image size");
  Allocator used;
  void* mem = dev_alloc(lay.total, p->stream, &used);
  if (!mem) return fail(PT_ENOMEM, "device allocation of %zu bytes failed", lay.total);
  p->dmem = mem;
  p->dbytes = lay.total;
  p->allocator_free = used.free;
  p->allocator_ctx = used.ctx;
  uint8_t* base = (uint8_t*)mem;
  DevProblem& d = p->dev;
  d.spins = (uint32_t*)(base + lay.spins);
  d.L = L;
  d.R = R;
  d.W = p->W;
  d.mode = p->mode;
  d.key0 = (uint32_t)seed;
  d.key1 = (uint32_t)(seed >> 32);
  d.table_shift = table_shift(Ji, hi);
  d.cmp_classes = 0;
  for (int kk = 0; kk <= 4; ++kk)
    for (int up = 0; up <= 1; ++up)
      if (2 * (Ji * (4 - 2 * kk) - hi * (up ? 1 : -1)) > 0) d.cmp_classes |= 1 << (2 * kk + up);
  d.J_int = Ji;
  d.h_int = hi;
  d.s = s;
  d.T_temp = (const uint64_t*)(base + lay.T_temp);
  d.planes = base + lay.planes;
  d.temp_of_slot = (int32_t*)(base + lay.temp_of_slot);
  d.slot_of_temp = (int32_t*)(base + lay.slot_of_temp);
  d.cnt = (uint32_t*)(base + lay.cnt);
  d.E_slot = (int64_t*)(base + lay.E_slot);
  d.M_slot = (int64_t*)(base + lay.M_slot);
  d.attempted = (uint64_t*)(base + lay.attempted);
  d.accepted = (uint64_t*)(base + lay.accepted);
  d.pairs = (const SwapPair*)(base + lay.pairs);
  d.swap_table = (const uint32_t*)(base + lay.table);
  d.status = (int32_t*)(base + lay.status);
#ifdef PT_DEBUG
  // the debug build's write tags (one per spin word) and check record, zeroed
  {
    const size_t tag_bytes = align256((size_t)p->W * L * L * 4);
    Allocator dused;
    void* dm = dev_alloc(tag_bytes + sizeof(DebugRecord), p->stream, &dused);
    if (!dm) {
      dev_free(mem, p->stream, used);
      return fail(PT_ENOMEM, "debug build: allocation of the write tags failed");
    }
    p->dbg_mem = dm;
    p->dbg_free = dused.free;
    p->dbg_ctx = dused.ctx;
    d.dbg_tag = (uint32_t*)dm;
    d.dbg = (DebugRecord*)((uint8_t*)dm + tag_bytes);
    if (cudaMemsetAsync(dm, 0, tag_bytes + sizeof(DebugRecord), p->stream) != cudaSuccess) {
      cudaGetLastError();
      dev_free(dm, p->stream, dused);
      dev_free(mem, p->stream, used);
      return fail(PT_ECUDA, "debug build: clearing the write tags failed");
    }
  }
#endif

  // one copy of the image (asynchronous from page-locked memory; from pageable memory the
  // call returns once the bytes are staged), the initial spins and the plane thresholds
  cudaError_t err = cudaMemcpyAsync(base + lay.T_temp, img->data(), img->bytes,
                                    cudaMemcpyHostToDevice, p->stream);
  if (err == cudaSuccess) err = launch_init(d, dev, p->stream);
  if (err == cudaSuccess) err = launch_exchange(d, 0, kStepRebuild, p->stream);
  if (err == cudaSuccess && !stream) err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(p->stream);
    cudaGetLastError();
    dev_free(mem, p->stream, used);
    if (p->dbg_mem) {
      Allocator da;
      da.free = p->dbg_free;
      da.ctx = p->dbg_ctx;
      dev_free(p->dbg_mem, p->stream, da);
    }
    return fail(PT_ECUDA, "initialising problem: %s", cudaGetErrorString(err));
  }
  if (img->locked) p->image = img;
  *out = p.release();
  return PT_OK;
}

void pt_destroy(pt_problem* p) {
  if (!p) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != p->dev_info.device) cudaSetDevice(p->dev_info.device);
  cudaStreamSynchronize(p->stream);
  cudaGetLastError();
  Allocator a;
  a.free = p->allocator_free;
  a.ctx = p->allocator_ctx;
  dev_free(p->dmem, p->stream, a);
  Allocator ta;
  ta.free = p->trace_free;
  ta.ctx = p->trace_ctx;
  dev_free(p->trace_mem, p->stream, ta);
  Allocator da;
  da.free = p->dbg_free;
  da.ctx = p->dbg_ctx;
  dev_free(p->dbg_mem, p->stream, da);
  Allocator ba;
  ba.free = p->band_free;
  ba.ctx = p->band_ctx;
  dev_free(p->band_mem, p->stream, ba);
  if (cur >= 0 && cur != p->dev_info.device) cudaSetDevice(cur);
  delete p;
}

int pt_set_stream(pt_problem* p, void* cuda_stream) {
  int rc = problem_check(p);
  if (rc) return rc;
  if ((rc = problem_device_guard(p))) return rc;
  const cudaError_t err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "synchronising old stream", err);
  p->stream = (cudaStream_t)cuda_stream;
  return PT_OK;
}

namespace {

// pt_sweep as cooperative launches of at most kPersistChunk sweeps each.
// The band form of the persistent kernel per sweep strategy: chosen where it measured
// faster (AUTO), never (PERSISTENT: the strided form), always (BANDS).
int band_choice(int strategy) {
  return strategy == PT_SWEEP_BANDS ? kBandForce
                                    : (strategy == PT_SWEEP_AUTO ? kBandAuto : kBandNever);
}

int sweep_persistent(pt_problem* p, int64_t n, int m) {
  if (p->plan.band && !p->band_mem) {
    // the band form's second copy of colour 1 (W L L/2 words), allocated once per problem
    Allocator used;
    void* mem = dev_alloc((size_t)p->W * p->L * (p->L / 2) * 4, p->stream, &used);
    if (!mem) return fail(PT_ENOMEM, "allocation of the band form's colour-1 copy failed");
    p->band_mem = mem;
    p->band_free = used.free;
    p->band_ctx = used.ctx;
    p->dev.band_c1 = (uint32_t*)mem;
  }
  while (n > 0) {
    const int c = (int)std::min<int64_t>(n, kPersistChunk);
    const cudaError_t err = launch_persist(p->dev, p->plan, p->t, p->e, c, m, p->stall,
                                           p->wait_limit_ns, p->stream);
    p->stall = 0;
    if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "persistent sweep launch", err);
    const uint64_t t1 = p->t + (uint64_t)c;
    if (m > 0) p->e += t1 / (uint64_t)m - p->t / (uint64_t)m;  // sweeps t with (t+1) % m == 0
    p->t = t1;
    n -= c;
  }
  return PT_OK;
}

}  // namespace

int pt_sweep(pt_problem* p, int64_t n, int exchange_every) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (n < 0 || exchange_every < 0)
    return fail(PT_EINVAL, "n = %lld and exchange_every = %d must be >= 0", (long long)n,
                exchange_every);
  if ((rc = problem_device_guard(p))) return rc;
  if (n == 0) return PT_OK;
  if (p->sweep_strategy != PT_SWEEP_LAUNCHES) {
    if (!p->plan_valid) {
      const cudaError_t err = persist_plan(p->dev, p->dev_info, p->words_per_thread,
                                           band_choice(p->sweep_strategy), &p->plan);
      if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "persistent occupancy", err);
      p->plan_valid = true;
    }
    if (p->plan.grid > 0) return sweep_persistent(p, n, exchange_every);
    if (p->sweep_strategy == PT_SWEEP_PERSISTENT || p->sweep_strategy == PT_SWEEP_BANDS)
      return fail(PT_EINVAL, "L = %d, R = %d does not fit one resident wave of the persistent "
                  "kernel with <= %d words per thread%s", p->L, p->R, kPersistMaxWordsPerThread,
                  p->sweep_strategy == PT_SWEEP_BANDS
                      ? " in bands of rows (at least two per plane, their copies within the "
                        "shared-memory limit)"
                      : "");
  }
  for (int64_t j = 0; j < n; ++j) {
    cudaError_t err = launch_half_sweep(p->dev, p->dev_info, 0, p->t, p->stream);
    p->dev.dbg_inject = 0;  // the debug build's test hook applies to one launch
    if (err == cudaSuccess) err = launch_half_sweep(p->dev, p->dev_info, 1, p->t, p->stream);
    if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "sweep launch", err);
    const bool ex = exchange_every > 0 && (p->t + 1) % (uint64_t)exchange_every == 0;
    const bool trace = p->dev.trace_E != nullptr;
    if (ex || trace) {
      const int flags = kStepEnergy | (ex ? kStepExchange | kStepRebuild : 0) |
                        (trace ? kStepTrace : 0);
      err = launch_energy(p->dev, p->dev_info, p->stream);
      if (err == cudaSuccess) err = launch_exchange(p->dev, p->e, flags, p->stream, p->t);
      if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "exchange launch", err);
      if (ex) p->e += 1;
    }
    p->t += 1;
  }
  return PT_OK;
}

int pt_flip(pt_problem* p, int64_t n, int exchange_every) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (n < 0 || exchange_every < 0)
    return fail(PT_EINVAL, "n = %lld and exchange_every = %d must be >= 0", (long long)n,
                exchange_every);
  if ((rc = problem_device_guard(p))) return rc;
  if (n == 0) return PT_OK;
  if ((rc = refresh_observables(p))) return rc;  // E_slot, M_slot of the current state
  const uint64_t m = (uint64_t)exchange_every;
  int k = 0;
  size_t smem = 0;
  if (p->flip_shared && (rc = flip_smem_plan(p->dev, p->dev_info.sms, p->dev_info.smem_optin,
                                             &k, &smem)))
    return fail(rc, "planning the shared-memory single-flip kernel");
  while (n > 0) {
    const int64_t c = std::min<int64_t>(n, (int64_t)1 << 24);
    const cudaError_t err =
        k > 0 ? launch_flip_smem(p->dev, k, smem, p->it, p->e, c, exchange_every, p->stall,
                                 p->wait_limit_ns, p->stream)
              : launch_flip(p->dev, p->it, p->e, c, exchange_every, p->stall, p->wait_limit_ns,
                            p->stream);
    p->stall = 0;
    if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "single-flip launch", err);
    const uint64_t it1 = p->it + (uint64_t)c;
    if (m > 0) p->e += it1 / m - p->it / m;
    p->it = it1;
    n -= c;
  }
  return PT_OK;
}

int pt_set_flip_tuning(pt_problem* p, int shared_memory) {
  int rc = problem_check(p);
  if (rc) return rc;
  p->flip_shared = shared_memory != 0;
  return PT_OK;
}

int pt_iterations(pt_problem* p, uint64_t* iterations_done) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (iterations_done) *iterations_done = p->it;
  return PT_OK;
}

int pt_set_sweep_tuning(pt_problem* p, int strategy, int words_per_thread) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (strategy < PT_SWEEP_AUTO || strategy > PT_SWEEP_BANDS)
    return fail(PT_EINVAL, "unknown sweep strategy %d", strategy);
  if (words_per_thread < 0 || words_per_thread > kPersistMaxWordsPerThread)
    return fail(PT_EINVAL, "words_per_thread = %d outside 0..%d", words_per_thread,
                kPersistMaxWordsPerThread);
  p->sweep_strategy = strategy;
  p->words_per_thread = words_per_thread ? words_per_thread : kPersistDefaultWords;
  p->plan_valid = false;
  return PT_OK;
}

int pt_get_sweep_tuning(pt_problem* p, int* strategy, int* words_per_thread, int* grid) {
  int rc = problem_check(p);
  if (rc) return rc;
  if ((rc = problem_device_guard(p))) return rc;
  if (!p->plan_valid) {
    const cudaError_t err = persist_plan(p->dev, p->dev_info, p->words_per_thread,
                                         band_choice(p->sweep_strategy), &p->plan);
    if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "persistent occupancy", err);
    p->plan_valid = true;
  }
  if (strategy) *strategy = p->sweep_strategy;
  if (words_per_thread) *words_per_thread = p->words_per_thread;
  if (grid) *grid = p->plan.grid;
  return PT_OK;
}

int pt_set_wait_limit(pt_problem* p, double seconds) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (!(seconds > 0.0 && seconds <= 60.0))
    return fail(PT_EINVAL, "wait limit %g s outside (0, 60]", seconds);
  p->wait_limit_ns = (uint64_t)(seconds * 1e9);
  return PT_OK;
}

int pt_debug_stall_barrier(pt_problem* p, int arrivals) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (arrivals < 0) return fail(PT_EINVAL, "arrivals = %d must be >= 0", arrivals);
  p->stall = arrivals;
  return PT_OK;
}

int pt_synchronize(pt_problem* p) {
  int rc = problem_check(p);
  if (rc) return rc;
  if ((rc = problem_device_guard(p))) return rc;
  cudaError_t err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "synchronise", err);
  int32_t status = 0;
  err = cudaMemcpy(&status, p->dev.status, 4, cudaMemcpyDeviceToHost);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "reading status", err);
  if (status != 0) {
    p->poisoned = status == PT_ETIMEOUT ? PT_ETIMEOUT : PT_EINTERNAL;
    return fail(p->poisoned, "device reported status %d%s", status,
                status == kStatusDebug ? " (a check of the debug build failed)" : "");
  }
  return PT_OK;
}

int pt_debug_build(void) { return PT_DBG_ON; }

int pt_debug_report(pt_problem* p, uint64_t* violations, int32_t* first_kind,
                    uint64_t* first_index, uint64_t* unwritten) {
  if (!p) return fail(PT_EINVAL, "problem is NULL");
  if (!PT_DBG_ON || !p->dbg_mem)
    return fail(PT_EINVAL, "pt_debug_report needs the debug build of the library");
  int rc = problem_device_guard(p);
  if (rc) return rc;
  cudaError_t err = cudaStreamSynchronize(p->stream);
  DebugRecord rec{};
  if (err == cudaSuccess)
    err = cudaMemcpy(&rec, p->dev.dbg, sizeof(DebugRecord), cudaMemcpyDeviceToHost);
  // the last sweep must have stored every word of colour c in half sweep 2 (t - 1) + c
  uint64_t missing = 0;
  if (err == cudaSuccess && p->t > p->dbg_t0) {
    const size_t n = (size_t)p->W * p->L * p->L;
    std::vector<uint32_t> tag(n);
    err = cudaMemcpy(tag.data(), p->dev.dbg_tag, n * 4, cudaMemcpyDeviceToHost);
    const size_t nc = (size_t)p->L * (p->L / 2);
    for (size_t g = 0; err == cudaSuccess && g < n; ++g) {
      const uint64_t c = (g / nc) & 1;
      const uint32_t want = (uint32_t)((2 * (p->t - 1) + c) % 0x7fffffffull) + 1u;
      missing += tag[g] != want;
    }
  }
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "reading the debug record", err);
  if (violations) *violations = rec.violations;
  if (first_kind) *first_kind = (int32_t)rec.first_kind;
  if (first_index) *first_index = rec.first_index;
  if (unwritten) *unwritten = missing;
  return PT_OK;
}

int pt_debug_inject(pt_problem* p, int kind) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (!PT_DBG_ON || !p->dbg_mem)
    return fail(PT_EINVAL, "pt_debug_inject needs the debug build of the library");
  if (kind < 0 || kind > 2) return fail(PT_EINVAL, "unknown planted mistake %d", kind);
  p->dev.dbg_inject = kind;
  return PT_OK;
}

int pt_energies_int(pt_problem* p, int64_t* E_int, int64_t* M, int64_t* scale) {
  int rc = problem_check(p);
  if (rc) return rc;
  if ((rc = problem_device_guard(p))) return rc;
  std::vector<int64_t> E, Ms;
  std::vector<int32_t> sot;
  if ((rc = read_observables(p, &E, &Ms, &sot))) return rc;
  for (int k = 0; k < p->R; ++k) {
    if (E_int) E_int[k] = E[sot[k]];
    if (M) M[k] = Ms[sot[k]];
  }
  if (scale) *scale = p->s;
  return pt_synchronize(p);
}

int pt_energies(pt_problem* p, double* out) {
  if (!out) return fail(PT_EINVAL, "out is NULL");
  std::vector<int64_t> E(p ? p->R : 0);
  int64_t s = 1;
  const int rc = pt_energies_int(p, E.data(), nullptr, &s);
  if (rc) return rc;
  for (int k = 0; k < p->R; ++k) out[k] = (double)E[k] / (double)s;
  return PT_OK;
}

int pt_magnetisations(pt_problem* p, double* out) {
  if (!out) return fail(PT_EINVAL, "out is NULL");
  std::vector<int64_t> M(p ? p->R : 0);
  const int rc = pt_energies_int(p, nullptr, M.data(), nullptr);
  if (rc) return rc;
  for (int k = 0; k < p->R; ++k) out[k] = (double)M[k];
  return PT_OK;
}

int pt_swap_stats(pt_problem* p, uint64_t* attempted, uint64_t* accepted) {
  int rc = problem_check(p);
  if (rc) return rc;
  if ((rc = problem_device_guard(p))) return rc;
  if (p->R < 2) return pt_synchronize(p);
  cudaError_t err = cudaSuccess;
  if (attempted)
    err = cudaMemcpyAsync(attempted, p->dev.attempted, (p->R - 1) * 8, cudaMemcpyDeviceToHost,
                          p->stream);
  if (err == cudaSuccess && accepted)
    err = cudaMemcpyAsync(accepted, p->dev.accepted, (p->R - 1) * 8, cudaMemcpyDeviceToHost,
                          p->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "reading swap stats", err);
  return pt_synchronize(p);
}

int pt_read_batch(pt_problem* const* ps, int count, int64_t* const* E_int, int64_t* const* M,
                  int32_t* const* slot_of_temp, uint64_t* const* attempted,
                  uint64_t* const* accepted) {
  if (count < 0 || (count > 0 && !ps)) return fail(PT_EINVAL, "count = %d, problems", count);
  if (count == 0) return PT_OK;
  cudaStream_t st = ps[0] ? ps[0]->stream : 0;
  for (int j = 0; j < count; ++j) {
    int rc = problem_check(ps[j]);
    if (rc) return rc;
    if (ps[j]->stream != st) return fail(PT_EINVAL, "problems of one read must share a stream");
    if (ps[j]->dev_info.device != ps[0]->dev_info.device)
      return fail(PT_EINVAL, "problems on different devices");
  }
  int rc = problem_device_guard(ps[0]);
  if (rc) return rc;
  // energies from the current spins (as the single getters): one count launch over every
  // problem's words and one gather that finishes the energies and packs the records, then
  // one copy. A problem listed more than once is read once (its counts are shared).
  std::vector<GatherItem> items;
  std::vector<EnergyChunk> chunks;
  std::vector<int64_t> rec_of((size_t)count);
  std::map<const pt_problem*, int64_t> seen;
  int64_t words = 0;
  for (int j = 0; j < count; ++j) {
    pt_problem* p = ps[j];
    auto dup = seen.find(p);
    if (dup != seen.end()) {
      rec_of[(size_t)j] = dup->second;
      continue;
    }
    seen.emplace(p, words);
    rec_of[(size_t)j] = words;
    const DevProblem& d = p->dev;
    items.emplace_back();
    GatherItem& it = items.back();
    it.E_slot = d.E_slot;
    it.M_slot = d.M_slot;
    it.slot_of_temp = d.slot_of_temp;
    it.attempted = d.attempted;
    it.accepted = d.accepted;
    it.status = d.status;
    it.cnt = d.cnt;
    it.J_int = d.J_int;
    it.h_int = d.h_int;
    it.L = d.L;
    it.W = d.W;
    it.R = p->R;
    it.npairs = p->R >= 2 ? p->R - 1 : 0;
    it.out = words;
    words += 1 + 3 * (int64_t)it.R + 2 * (int64_t)it.npairs;
    const int nwords = d.L * (d.L >> 1);
    for (int w = 0; w < d.W; ++w)
      for (int first = 0; first < nwords; first += kEnergyChunkWords)
        chunks.push_back(EnergyChunk{d.spins, d.cnt, d.L, d.W, w, first,
                                     std::min(kEnergyChunkWords, nwords - first), d.dbg,
                                     d.status});
  }
  if (chunks.size() > (size_t)INT32_MAX) return fail(PT_EINVAL, "batched read too large");
  const int nitems = (int)items.size();
  const size_t ib = ((size_t)nitems * sizeof(GatherItem) + 255) & ~size_t(255);
  const size_t cb = (chunks.size() * sizeof(EnergyChunk) + 255) & ~size_t(255);
  std::vector<uint8_t> staging(ib + cb);
  memcpy(staging.data(), items.data(), (size_t)nitems * sizeof(GatherItem));
  memcpy(staging.data() + ib, chunks.data(), chunks.size() * sizeof(EnergyChunk));
  void* scratch = nullptr;
  cudaError_t err = cudaMallocAsync(&scratch, ib + cb + (size_t)words * 8, st);
  if (err != cudaSuccess) return fail(PT_ENOMEM, "read scratch: %s", cudaGetErrorString(err));
  GatherItem* d_items = (GatherItem*)scratch;
  EnergyChunk* d_chunks = (EnergyChunk*)((char*)scratch + ib);
  uint64_t* d_out = (uint64_t*)((char*)scratch + ib + cb);
  std::vector<uint64_t> host((size_t)words);
  err = cudaMemcpyAsync(scratch, staging.data(), staging.size(), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = launch_energy_batch(d_chunks, (int)chunks.size(), st);
  if (err == cudaSuccess) err = launch_gather(d_items, nitems, d_out, ps[0]->dev_info.sms, st);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(host.data(), d_out, (size_t)words * 8, cudaMemcpyDeviceToHost, st);
  const cudaError_t err2 = cudaFreeAsync(scratch, st);
  if (err == cudaSuccess) err = err2;
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) {
    for (int j = 0; j < count; ++j) ps[j]->poisoned = PT_ECUDA;
    return fail(PT_ECUDA, "batched read: %s", cudaGetErrorString(err));
  }
  int first_rc = PT_OK;
  for (int j = 0; j < count; ++j) {
    pt_problem* p = ps[j];
    const uint64_t* rec = host.data() + rec_of[(size_t)j];
    const int R = p->R, P = R >= 2 ? R - 1 : 0;
    const int32_t status = (int32_t)(int64_t)rec[0];
    if (status != 0) {
      p->poisoned = status == PT_ETIMEOUT ? PT_ETIMEOUT : PT_EINTERNAL;
      if (first_rc == PT_OK)
        first_rc = fail(p->poisoned, "problem %d: device reported status %d", j, status);
      continue;
    }
    const uint64_t* E = rec + 1;
    const uint64_t* Ms = rec + 1 + R;
    const uint64_t* sot = rec + 1 + 2 * R;
    for (int k = 0; k < R; ++k) {
      const int a = (int)(int64_t)sot[k];
      if (E_int && E_int[j]) E_int[j][k] = (int64_t)E[a];
      if (M && M[j]) M[j][k] = (int64_t)Ms[a];
      if (slot_of_temp && slot_of_temp[j]) slot_of_temp[j][k] = a;
    }
    for (int k = 0; k < P; ++k) {
      if (attempted && attempted[j]) attempted[j][k] = rec[1 + 3 * R + k];
      if (accepted && accepted[j]) accepted[j][k] = rec[1 + 3 * R + P + k];
    }
  }
  return first_rc;
}

int pt_chain_map(pt_problem* p, int32_t* slot_of_temp) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (!slot_of_temp) return fail(PT_EINVAL, "out is NULL");
  if ((rc = problem_device_guard(p))) return rc;
  cudaError_t err = cudaMemcpyAsync(slot_of_temp, p->dev.slot_of_temp, p->R * 4,
                                    cudaMemcpyDeviceToHost, p->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "reading chain map", err);
  return pt_synchronize(p);
}

int pt_temperature_map(pt_problem* p, int32_t* slot_of_temp) {
  return pt_chain_map(p, slot_of_temp);
}

int pt_counters(pt_problem* p, uint64_t* sweeps_done, uint64_t* exchanges_done) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (sweeps_done) *sweeps_done = p->t;
  if (exchanges_done) *exchanges_done = p->e;
  return PT_OK;
}

size_t pt_device_bytes(const pt_problem* p) { return p ? p->dbytes + p->trace_bytes : 0; }

size_t pt_checkpoint_bytes(const pt_problem* p) { return p ? ckpt_bytes(p->L, p->R) : 0; }

int pt_save(pt_problem* p, void* buf, size_t bytes) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (!buf) return fail(PT_EINVAL, "buf is NULL");
  const size_t need = ckpt_bytes(p->L, p->R);
  if (bytes < need) return fail(PT_EINVAL, "checkpoint needs %zu bytes, got %zu", need, bytes);
  if ((rc = problem_device_guard(p))) return rc;
  const int R = p->R, W = p->W;
  const size_t pairs = (size_t)std::max(R - 1, 0);
  std::vector<int32_t> sot((size_t)R);
  std::vector<uint64_t> att(pairs), acc(pairs);
  uint8_t* out = (uint8_t*)buf;
  const size_t spin_off = kCkptHeader + (size_t)R * 12 + pairs * 16;
  cudaError_t err = cudaMemcpyAsync(sot.data(), p->dev.slot_of_temp, (size_t)R * 4,
                                    cudaMemcpyDeviceToHost, p->stream);
  if (err == cudaSuccess && pairs) {
    err = cudaMemcpyAsync(att.data(), p->dev.attempted, pairs * 8, cudaMemcpyDeviceToHost,
                          p->stream);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(acc.data(), p->dev.accepted, pairs * 8, cudaMemcpyDeviceToHost,
                            p->stream);
  }
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(out + spin_off, p->dev.spins, (size_t)W * p->L * p->L * 4,
                          cudaMemcpyDeviceToHost, p->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "reading the checkpoint", err);
  if ((rc = pt_synchronize(p))) return rc;
  Writer w{out};
  w.put_bytes(kCkptMagic, 8);
  w.put((uint32_t)p->L);
  w.put((uint32_t)p->R);
  w.put(p->J);
  w.put(p->h);
  w.put(p->seed);
  w.put(p->t);
  w.put(p->e);
  w.put((int32_t)p->swap_rule);
  w.put((int32_t)0);
  w.put(p->it);
  w.put_bytes(p->betas.data(), (size_t)R * 8);
  w.put_bytes(sot.data(), (size_t)R * 4);
  if (pairs) {
    w.put_bytes(att.data(), pairs * 8);
    w.put_bytes(acc.data(), pairs * 8);
  }
  const uint64_t sum = fnv1a64(out, need - 8);
  memcpy(out + need - 8, &sum, 8);
  return PT_OK;
}

int pt_load(const void* buf, size_t bytes, pt_problem** out) {
  if (!out) return fail(PT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!buf || bytes < kCkptHeader + 8) return fail(PT_EINVAL, "checkpoint too short");
  const uint8_t* in = (const uint8_t*)buf;
  if (memcmp(in, kCkptMagic, 8) != 0) return fail(PT_EINVAL, "not a checkpoint (magic)");
  Reader r{in + 8};
  const uint32_t L = r.get<uint32_t>(), R = r.get<uint32_t>();
  const double J = r.get<double>(), h = r.get<double>();
  const uint64_t seed = r.get<uint64_t>(), t = r.get<uint64_t>(), e = r.get<uint64_t>();
  const int32_t rule = r.get<int32_t>();
  r.get<int32_t>();
  const uint64_t it = r.get<uint64_t>();
  if (L < 4 || L > PT_MAX_L || (L & 1) || R < 1 || R > PT_MAX_R)
    return fail(PT_EINVAL, "checkpoint with L = %u, R = %u", L, R);
  const size_t need = ckpt_bytes((int)L, (int)R);
  if (bytes != need) return fail(PT_EINVAL, "checkpoint of %zu bytes, expected %zu", bytes, need);
  uint64_t sum;
  memcpy(&sum, in + need - 8, 8);
  if (sum != fnv1a64(in, need - 8)) return fail(PT_EINVAL, "checkpoint checksum mismatch");
  if (rule != PT_SWAP_BARKER && rule != PT_SWAP_METROPOLIS)
    return fail(PT_EINVAL, "checkpoint with swap rule %d", rule);
  const int W = ((int)R + 31) / 32;
  const size_t pairs = (size_t)R - 1;
  std::vector<double> betas(R);
  std::vector<int32_t> sot(R);
  std::vector<uint64_t> att(pairs), acc(pairs);
  const uint8_t* q = in + kCkptHeader;
  memcpy(betas.data(), q, (size_t)R * 8);
  q += (size_t)R * 8;
  memcpy(sot.data(), q, (size_t)R * 4);
  q += (size_t)R * 4;
  if (pairs) {
    memcpy(att.data(), q, pairs * 8);
    memcpy(acc.data(), q + pairs * 8, pairs * 8);
  }
  q += pairs * 16;
  // the map must be a permutation; the counters consistent
  std::vector<int32_t> tos(R, -1);
  for (uint32_t k = 0; k < R; ++k) {
    if (sot[k] < 0 || sot[k] >= (int32_t)R || tos[sot[k]] >= 0)
      return fail(PT_EINVAL, "checkpoint temperature map is not a permutation");
    tos[sot[k]] = (int32_t)k;
  }
  for (size_t k = 0; k < pairs; ++k)
    if (acc[k] > att[k]) return fail(PT_EINVAL, "checkpoint pair %zu: accepted > attempted", k);
  // unused bits of the last plane are zero
  const int last = (int)R - 32 * (W - 1);
  if (last < 32) {
    const uint32_t unused = ~((1u << last) - 1u);
    const size_t words = (size_t)L * L;
    for (size_t i = 0; i < words; ++i) {
      uint32_t v;
      memcpy(&v, q + ((size_t)(W - 1) * words + i) * 4, 4);
      if (v & unused) return fail(PT_EINVAL, "checkpoint sets bits of unused slots");
    }
  }
  pt_options opt{};
  opt.size = sizeof opt;
  opt.swap_rule = rule;
  pt_problem* p = nullptr;
  int rc = pt_create_ex((int)L, betas.data(), (int)R, J, h, seed, &opt, &p);
  if (rc) return rc;
  cudaError_t err = cudaMemcpyAsync(p->dev.spins, q, (size_t)W * L * L * 4,
                                    cudaMemcpyHostToDevice, p->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(p->dev.slot_of_temp, sot.data(), (size_t)R * 4,
                          cudaMemcpyHostToDevice, p->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(p->dev.temp_of_slot, tos.data(), (size_t)R * 4,
                          cudaMemcpyHostToDevice, p->stream);
  if (err == cudaSuccess && pairs) {
    err = cudaMemcpyAsync(p->dev.attempted, att.data(), pairs * 8, cudaMemcpyHostToDevice,
                          p->stream);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(p->dev.accepted, acc.data(), pairs * 8, cudaMemcpyHostToDevice,
                            p->stream);
  }
  if (err == cudaSuccess) err = launch_exchange(p->dev, 0, kStepRebuild, p->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) {
    cudaGetLastError();
    pt_destroy(p);
    return fail(PT_ECUDA, "restoring the checkpoint: %s", cudaGetErrorString(err));
  }
  p->t = t;
  p->e = e;
  p->it = it;
  p->dbg_t0 = t;  // the debug build's tags start with the next sweep
  *out = p;
  return PT_OK;
}

int pt_trace_start(pt_problem* p, int64_t capacity) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (capacity < 1 || capacity > ((int64_t)1 << 32))
    return fail(PT_EINVAL, "trace capacity %lld outside [1, 2^32]", (long long)capacity);
  if ((rc = problem_device_guard(p))) return rc;
  if ((rc = pt_trace_stop(p))) return rc;
  const size_t bytes = (size_t)capacity * p->R * 2 * sizeof(int64_t);
  Allocator used;
  void* mem = dev_alloc(bytes, p->stream, &used);
  if (!mem) return fail(PT_ENOMEM, "trace ring of %zu bytes", bytes);
  const cudaError_t err = cudaMemsetAsync(mem, 0, bytes, p->stream);
  if (err != cudaSuccess) {
    dev_free(mem, p->stream, used);
    return problem_fail(p, PT_ECUDA, "clearing the trace ring", err);
  }
  p->trace_mem = mem;
  p->trace_bytes = bytes;
  p->trace_free = used.free;
  p->trace_ctx = used.ctx;
  p->dev.trace_E = (int64_t*)mem;
  p->dev.trace_M = (int64_t*)mem + (size_t)capacity * p->R;
  p->dev.trace_cap = capacity;
  p->dev.trace_t0 = p->t;
  return PT_OK;
}

int pt_trace_stop(pt_problem* p) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (!p->trace_mem) return PT_OK;
  if ((rc = problem_device_guard(p))) return rc;
  const cudaError_t err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "synchronise", err);
  Allocator a;
  a.free = p->trace_free;
  a.ctx = p->trace_ctx;
  dev_free(p->trace_mem, p->stream, a);
  p->trace_mem = nullptr;
  p->trace_bytes = 0;
  p->dev.trace_E = p->dev.trace_M = nullptr;
  p->dev.trace_cap = 0;
  return PT_OK;
}

int pt_trace_read(pt_problem* p, int64_t max_rows, int64_t* E_int, int64_t* M,
                  uint64_t* first_sweep, int64_t* rows) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (max_rows < 0) return fail(PT_EINVAL, "max_rows = %lld", (long long)max_rows);
  if (!p->trace_mem) return fail(PT_ESTATE, "no trace: call pt_trace_start first");
  if ((rc = problem_device_guard(p))) return rc;
  const int64_t written = (int64_t)(p->t - p->dev.trace_t0);
  const int64_t n = std::min<int64_t>(std::min<int64_t>(written, p->dev.trace_cap), max_rows);
  const uint64_t first = p->t - (uint64_t)n;  // sweep index (0-based) of the first row
  const int R = p->R;
  cudaError_t err = cudaSuccess;
  // rows first .. first + n - 1, in at most two pieces of the ring
  int64_t done = 0;
  while (done < n && err == cudaSuccess) {
    const int64_t slot = (int64_t)((first + done - p->dev.trace_t0) % (uint64_t)p->dev.trace_cap);
    const int64_t len = std::min<int64_t>(n - done, p->dev.trace_cap - slot);
    const size_t off = (size_t)slot * R, cnt = (size_t)len * R * sizeof(int64_t);
    if (E_int)
      err = cudaMemcpyAsync(E_int + (size_t)done * R, p->dev.trace_E + off, cnt,
                            cudaMemcpyDeviceToHost, p->stream);
    if (err == cudaSuccess && M)
      err = cudaMemcpyAsync(M + (size_t)done * R, p->dev.trace_M + off, cnt,
                            cudaMemcpyDeviceToHost, p->stream);
    done += len;
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "reading the trace", err);
  if (first_sweep) *first_sweep = first + 1;
  if (rows) *rows = n;
  return pt_synchronize(p);
}

int pt_get_spins(pt_problem* p, int k, int8_t* out) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (!out || k < 0 || k >= p->R) return fail(PT_EINVAL, "bad temperature index %d", k);
  if ((rc = problem_device_guard(p))) return rc;
  int r;
  if ((rc = slot_at_temperature(p, k, &r))) return rc;
  std::vector<uint32_t> plane;
  if ((rc = read_plane(p, r >> 5, &plane))) return rc;
  const int L = p->L, half = L / 2, b = r & 31;
  for (int c = 0; c < 2; ++c)
    for (int y = 0; y < L; ++y)
      for (int i = 0; i < half; ++i) {
        const int x = 2 * i + ((y + c) & 1);
        const uint32_t w = plane[((size_t)c * L + y) * half + i];
        out[(size_t)y * L + x] = ((w >> b) & 1u) ? (int8_t)1 : (int8_t)-1;
      }
  return pt_synchronize(p);
}

int pt_set_spins(pt_problem* p, int k, const int8_t* in) {
  int rc = problem_check(p);
  if (rc) return rc;
  if (!in || k < 0 || k >= p->R) return fail(PT_EINVAL, "bad temperature index %d", k);
  const int L = p->L, half = L / 2;
  for (size_t q = 0; q < (size_t)L * L; ++q)
    if (in[q] != 1 && in[q] != -1) return fail(PT_EINVAL, "spin %zu is %d, not +-1", q, in[q]);
  if ((rc = problem_device_guard(p))) return rc;
  int r;
  if ((rc = slot_at_temperature(p, k, &r))) return rc;
  std::vector<uint32_t> plane;
  if ((rc = read_plane(p, r >> 5, &plane))) return rc;
  const int b = r & 31;
  for (int c = 0; c < 2; ++c)
    for (int y = 0; y < L; ++y)
      for (int i = 0; i < half; ++i) {
        const int x = 2 * i + ((y + c) & 1);
        uint32_t& w = plane[((size_t)c * L + y) * half + i];
        w = (w & ~(1u << b)) | ((in[(size_t)y * L + x] > 0 ? 1u : 0u) << b);
      }
  cudaError_t err = cudaMemcpyAsync(p->dev.spins + (size_t)(r >> 5) * L * L, plane.data(),
                                    plane.size() * 4, cudaMemcpyHostToDevice, p->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(p->stream);
  if (err != cudaSuccess) return problem_fail(p, PT_ECUDA, "writing spins", err);
  return PT_OK;
}

int pt_set_batch_tuning(int strategy, int cluster, int joint_min_L) {
  if ((strategy != PT_BATCH_FLAT && strategy != PT_BATCH_CLUSTER && strategy != PT_BATCH_FLOW &&
       strategy != PT_BATCH_QUEUE) ||
      cluster < 1 ||
      cluster > 16 || joint_min_L < 4)
    return fail(PT_EINVAL, "strategy = %d, cluster = %d, joint_min_L = %d", strategy, cluster,
                joint_min_L);
  std::lock_guard<std::mutex> lk(g_mu);
  g_batch_tuning.strategy = strategy;
  g_batch_tuning.cluster = cluster;
  g_batch_tuning.joint_min_L = joint_min_L;
  return PT_OK;
}

int pt_set_batch_tile_words(int tile_words) {
  if (tile_words < PT_TILE_WORDS_MIN || tile_words > PT_TILE_WORDS_MAX || tile_words % 32 != 0)
    return fail(PT_EINVAL, "tile_words = %d (a multiple of 32 in [%d, %d])", tile_words,
                PT_TILE_WORDS_MIN, PT_TILE_WORDS_MAX);
  std::lock_guard<std::mutex> lk(g_mu);
  g_batch_tuning.tile_words = tile_words;
  return PT_OK;
}

int pt_set_batch_streams(int streams) {
  if (streams < 1 || streams > PT_BATCH_STREAMS_MAX)
    return fail(PT_EINVAL, "streams = %d outside 1..%d", streams, PT_BATCH_STREAMS_MAX);
  std::lock_guard<std::mutex> lk(g_mu);
  g_batch_tuning.streams = streams;
  return PT_OK;
}

int pt_get_batch_streams(int* streams) {
  if (!streams) return fail(PT_EINVAL, "null output");
  std::lock_guard<std::mutex> lk(g_mu);
  *streams = g_batch_tuning.streams;
  return PT_OK;
}

int pt_set_batch_graphs(int on) {
  if (on != 0 && on != 1) return fail(PT_EINVAL, "graphs = %d: 0 or 1", on);
  std::lock_guard<std::mutex> lk(g_mu);
  g_batch_tuning.graphs = on;
  return PT_OK;
}

int pt_get_batch_graphs(int* on) {
  if (!on) return fail(PT_EINVAL, "null output");
  std::lock_guard<std::mutex> lk(g_mu);
  *on = g_batch_tuning.graphs;
  return PT_OK;
}

int pt_get_batch_tile_words(int* tile_words) {
  if (!tile_words) return fail(PT_EINVAL, "null output");
  std::lock_guard<std::mutex> lk(g_mu);
  *tile_words = g_batch_tuning.tile_words;
  return PT_OK;
}

int pt_get_batch_tuning(int* strategy, int* cluster, int* joint_min_L) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (strategy) *strategy = g_batch_tuning.strategy;
  if (cluster) *cluster = g_batch_tuning.cluster;
  if (joint_min_L) *joint_min_L = g_batch_tuning.joint_min_L;
  return PT_OK;
}

int pt_sweep_batch(pt_problem* const* problems, int count, const int64_t* n,
                   const int* exchange_every) {
  if (count < 0 || (count > 0 && (!problems || !n || !exchange_every)))
    return fail(PT_EINVAL, "bad batch arguments");
  if (count == 0) return PT_OK;
  return ptb::sweep_batch(problems, count, n, exchange_every);
}

int pt_sweep_batch_static(pt_problem* const* problems, int count, const int64_t* n,
                          const int* exchange_every) {
  if (count < 0 || (count > 0 && (!problems || !n || !exchange_every)))
    return fail(PT_EINVAL, "bad batch arguments");
  if (count == 0) return PT_OK;
  return ptb::sweep_batch_static_entry(problems, count, n, exchange_every);
}

}  // extern "C"
