// C-ABI entry points (include/rel.h): argument validation, planning, the
// mapping of a descriptor onto a specialised kernel, and the launches.
// Validation happens before any CUDA call, so a rejected request never
// touches the device.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "distinct.cuh"
#include "groupby.cuh"
#include "join.cuh"
#include "mlp.cuh"
#include "sketch.cuh"

#include <cmath>

// ------------------------------------------------------------ host helpers

namespace relhost {

static thread_local char g_err[512] = "";
static std::atomic<uint64_t> g_launches{0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

rel_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return REL_E_CUDA;
}

void count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Event timing of launches (rel_profile_start / rel_profile_stop).
struct ProfRec {
  int id;
  cudaEvent_t a, b;
};
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;      // records of the current window
static std::vector<cudaEvent_t> g_pool;  // events reused across windows
static size_t g_pool_used = 0;

static cudaEvent_t pool_event() {
  if (g_pool_used == g_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_pool.push_back(e);
  }
  return g_pool[g_pool_used++];
}

void launch_begin(int id, cudaStream_t st) {
  count_launch(1);
  if (!g_prof_on) return;
  ProfRec r{id, pool_event(), pool_event()};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, st);
  g_prof.push_back(r);
}

void launch_end(int id, cudaStream_t st) {
  if (!g_prof_on || g_prof.empty() || g_prof.back().id != id) return;
  cudaEventRecord(g_prof.back().b, st);
}

int device_sms() {
  static int cache[128] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return 148;
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 148;
    cache[dev] = n;
  }
  return cache[dev];
}

}  // namespace relhost

using relhost::set_error;

namespace {

using namespace rel;

constexpr int32_t TABLE_MAGIC = 0x4a4f494e;  // "JOIN"
constexpr int64_t MAX_INDEX_ROWS = 2147483647;

int elem_size(int32_t t) { return t == REL_U8 ? 1 : t == REL_I32 ? 4 : 8; }
int elem_bits(int32_t t) { return 8 * elem_size(t); }
bool valid_type(int32_t t) { return t == REL_U8 || t == REL_I32 || t == REL_I64; }

int log2_pow2(uint64_t x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

rel_status validate_desc(const rel_groupby_desc* d) {
  if (!d) return set_error("group-by: NULL descriptor"), REL_E_INVALID;
  if (d->n_rows < 0) return set_error("group-by: n_rows < 0"), REL_E_INVALID;
  if (d->n_cols < 1 || d->n_cols > REL_MAX_COLS || !d->cols)
    return set_error("group-by: n_cols must be 1..%d", REL_MAX_COLS), REL_E_INVALID;
  for (int c = 0; c < d->n_cols; ++c) {
    if (!valid_type(d->cols[c].type))
      return set_error("group-by: column %d has an unknown type", c), REL_E_INVALID;
    if (d->n_rows > 0 && !d->cols[c].data)
      return set_error("group-by: column %d has no data", c), REL_E_INVALID;
    if ((uintptr_t)d->cols[c].data % elem_size(d->cols[c].type))
      return set_error("group-by: column %d is not aligned to its element", c), REL_E_INVALID;
  }
  auto col_ok = [&](int32_t c) { return c >= 0 && c < d->n_cols; };
  if (d->n_keys < 1 || d->n_keys > REL_MAX_KEYS || !d->key_cols)
    return set_error("group-by: n_keys must be 1..%d", REL_MAX_KEYS), REL_E_INVALID;
  int bits = 0;
  for (int k = 0; k < d->n_keys; ++k) {
    if (!col_ok(d->key_cols[k])) return set_error("group-by: bad key column"), REL_E_INVALID;
    int32_t t = d->cols[d->key_cols[k]].type;
    if (d->n_keys > 1 && t == REL_I64)
      return set_error("group-by: a packed key may not contain an int64 column"), REL_E_INVALID;
    bits += elem_bits(t);
  }
  if (d->n_keys > 1 && bits > 64)
    return set_error("group-by: packed key wider than 64 bits"), REL_E_INVALID;
  if (d->n_preds < 0 || d->n_preds > REL_MAX_PREDS || (d->n_preds && !d->preds))
    return set_error("group-by: n_preds must be 0..%d", REL_MAX_PREDS), REL_E_INVALID;
  for (int i = 0; i < d->n_preds; ++i)
    if (!col_ok(d->preds[i].col)) return set_error("group-by: bad predicate column"), REL_E_INVALID;
  if (d->n_aggs < 1 || d->n_aggs > REL_MAX_AGGS || !d->aggs)
    return set_error("group-by: n_aggs must be 1..%d", REL_MAX_AGGS), REL_E_INVALID;
  for (int a = 0; a < d->n_aggs; ++a) {
    const rel_agg& g = d->aggs[a];
    if (g.op < REL_SUM || g.op > REL_MAX) return set_error("group-by: bad aggregate op"), REL_E_INVALID;
    if (g.op == REL_COUNT) continue;
    if (!col_ok(g.base_col)) return set_error("group-by: bad aggregate column"), REL_E_INVALID;
    if (g.nf < 0 || g.nf > 2) return set_error("group-by: nf must be 0..2"), REL_E_INVALID;
    for (int f = 0; f < g.nf; ++f)
      if (!col_ok(g.fcol[f])) return set_error("group-by: bad factor column"), REL_E_INVALID;
  }
  return REL_OK;
}

struct HostHeader {
  unsigned long long n_out, n_side;
  unsigned int overflow, timeout;
  unsigned long long aux;
};

rel_status read_header(const void* ws, HostHeader* h, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(h, ws, sizeof(HostHeader), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "reading the status header");
}

// A descriptor mapped onto a kernel shape.  perm[a] is the user aggregate
// that kernel word a computes (the KV shapes hold their words in a fixed
// internal order).
struct Mapped {
  int shape = SHAPE_GENERIC;
  int perm[REL_MAX_AGGS];
};

Mapped match_shape(const rel_groupby_desc* d, GbParams& p) {
  Mapped m;
  for (int a = 0; a < REL_MAX_AGGS; ++a) m.perm[a] = a;
  auto T = [&](int c) { return d->cols[c].type; };
  // key column + one int64 value column, no filter, no factors
  if (d->n_keys == 1 && d->n_preds == 0 && d->n_aggs <= 4 &&
      (T(d->key_cols[0]) == REL_I64 || T(d->key_cols[0]) == REL_I32)) {
    int vcol = -1;
    bool ok = true;
    int at[4] = {-1, -1, -1, -1};  // user index of SUM, COUNT, MIN, MAX
    bool dup = false;
    for (int a = 0; a < d->n_aggs && ok; ++a) {
      const rel_agg& g = d->aggs[a];
      const int slot = g.op == REL_SUM ? 0 : g.op == REL_COUNT ? 1 : g.op == REL_MIN ? 2 : 3;
      if (at[slot] >= 0) dup = true;
      at[slot] = a;
      if (g.op == REL_COUNT) continue;
      if (g.nf != 0 || T(g.base_col) != REL_I64) ok = false;
      else if (vcol < 0) vcol = g.base_col;
      else if (vcol != g.base_col) ok = false;
    }
    if (ok && vcol >= 0) {
      p.r_a = vcol;
      const bool k64 = T(d->key_cols[0]) == REL_I64;
      if (!dup && d->n_aggs == 4) {
        for (int i = 0; i < 4; ++i) m.perm[i] = at[i];
        m.shape = k64 ? SHAPE_KV4_64 : SHAPE_KV4_32;
      } else if (!dup && d->n_aggs == 2 && at[0] >= 0 && at[1] >= 0) {
        m.perm[0] = at[0];
        m.perm[1] = at[1];
        m.shape = k64 ? SHAPE_KV2_64 : SHAPE_KV2_32;
      } else {
        m.shape = k64 ? SHAPE_KVRT64 : SHAPE_KVRT32;
      }
      return m;
    }
  }
  // (u8, u8) key, one int32 range filter, five aggregates of the form
  // sum(a), sum(b), sum(b*f0(d)), sum(b*f0(d)*f1(t)), count over int64 columns
  if (d->n_keys == 2 && T(d->key_cols[0]) == REL_U8 && T(d->key_cols[1]) == REL_U8 &&
      d->n_preds == 1 && T(d->preds[0].col) == REL_I32 && d->n_aggs == 5) {
    const rel_agg* g = d->aggs;
    auto i64 = [&](int c) { return T(c) == REL_I64; };
    const bool ok = g[0].op == REL_SUM && g[0].nf == 0 && i64(g[0].base_col) &&
                    g[1].op == REL_SUM && g[1].nf == 0 && i64(g[1].base_col) &&
                    g[2].op == REL_SUM && g[2].nf == 1 && g[2].base_col == g[1].base_col &&
                    i64(g[2].fcol[0]) && g[3].op == REL_SUM && g[3].nf == 2 &&
                    g[3].base_col == g[1].base_col && g[3].fcol[0] == g[2].fcol[0] &&
                    g[3].c[0] == g[2].c[0] && g[3].s[0] == g[2].s[0] && i64(g[3].fcol[1]) &&
                    g[4].op == REL_COUNT;
    if (ok) {
      p.r_k0 = d->key_cols[0];
      p.r_k1 = d->key_cols[1];
      p.r_pred = d->preds[0].col;
      p.r_a = g[0].base_col;
      p.r_b = g[1].base_col;
      p.r_d = g[2].fcol[0];
      p.r_t = g[3].fcol[1];
      m.shape = SHAPE_Q1;
    }
  }
  return m;
}

// Kernel parameters of a descriptor, aggregates in the mapped order.
void fill_params(const rel_groupby_desc* d, const int* perm, GbParams& p) {
  std::memset(&p, 0, sizeof p);
  p.wait_ns = WAIT_LIMIT_NS;
  p.n_rows = d->n_rows;
  p.n_cols = d->n_cols;
  p.n_keys = d->n_keys;
  p.n_preds = d->n_preds;
  p.n_aggs = d->n_aggs;
  for (int c = 0; c < d->n_cols; ++c) {
    p.col[c] = (const uint8_t*)d->cols[c].data;
    p.ctype[c] = d->cols[c].type;
    p.csize[c] = elem_size(d->cols[c].type);
  }
  int shift = 0;
  for (int k = d->n_keys - 1; k >= 0; --k) {
    const int w = elem_bits(d->cols[d->key_cols[k]].type);
    p.key_col[k] = d->key_cols[k];
    p.key_shift[k] = d->n_keys == 1 ? 0 : shift;
    p.key_mask[k] = w >= 64 ? ~0ull : ((1ull << w) - 1);
    shift += w;
  }
  for (int i = 0; i < d->n_preds; ++i) {
    p.pred_col[i] = d->preds[i].col;
    p.pred_lo[i] = d->preds[i].lo;
    p.pred_hi[i] = d->preds[i].hi;
  }
  for (int a = 0; a < d->n_aggs; ++a) {
    const rel_agg& g = d->aggs[perm[a]];
    p.aop[a] = g.op;
    p.abase[a] = g.op == REL_COUNT ? 0 : g.base_col;
    p.anf[a] = g.op == REL_COUNT ? 0 : g.nf;
    for (int f = 0; f < 2; ++f) {
      p.afcol[a][f] = f < p.anf[a] ? g.fcol[f] : 0;
      p.ac[a][f] = g.c[f];
      p.as[a][f] = g.s[f];
    }
    if (agg_kind(g.op) == KIND_UMAX) p.umax_mask |= 1u << a;
  }
}

void set_stages(GbParams& p, int tile, int stages) {
  p.tile_rows = tile;
  p.n_stages = stages;
  uint32_t off = 0;
  for (int c = 0; c < p.n_cols; ++c) {
    p.stage_off[c] = off;
    off += (uint32_t)(tile * p.csize[c]);  // multiple of 16: tile % 16 == 0
  }
  p.stage_bytes = off;
}

bool tma_ok(const GbParams& p) {
  for (int c = 0; c < p.n_cols; ++c)
    if ((uintptr_t)p.col[c] % 16) return false;
  return true;
}

// Occupancy of each configuration, cached (the occupancy query is not free).
struct OccKey {
  int shape, mode, tma;
  uint32_t tiny, shared, tile, stages, stage_bytes;
  bool operator<(const OccKey& o) const {
    return std::tie(shape, mode, tma, tiny, shared, tile, stages, stage_bytes) <
           std::tie(o.shape, o.mode, o.tma, o.tiny, o.shared, o.tile, o.stages, o.stage_bytes);
  }
};
std::mutex g_occ_mu;
std::map<OccKey, int> g_occ[64];

int cached_occupancy(GbParams& p, int shape, int mode, bool tma) {
  int dev = 0;
  cudaGetDevice(&dev);
  dev &= 63;
  const OccKey k{shape, mode, tma, p.tiny_slots, p.smem_slots, (uint32_t)p.tile_rows,
                 (uint32_t)p.n_stages, p.stage_bytes};
  {
    std::lock_guard<std::mutex> lock(g_occ_mu);
    auto it = g_occ[dev].find(k);
    if (it != g_occ[dev].end()) return it->second;
  }
  const int occ = gb_ctas_per_sm(p, shape, mode, tma);
  std::lock_guard<std::mutex> lock(g_occ_mu);
  g_occ[dev][k] = occ;
  return occ;
}

// Pick rows per tile and ring depth: enough bytes in flight per SM to cover
// HBM latency (>= 64 KB), then as many resident warps as possible.
bool configure_stages(GbParams& p, int shape, int mode, bool tma) {
  if (!tma) {
    set_stages(p, 1024, 2);
    return cached_occupancy(p, shape, mode, false) > 0;
  }
  if (p.req_tile && p.req_stages) {  // the plan (an autotuner) chose
    const int t = p.req_tile, ns = p.req_stages;
    set_stages(p, t, ns);
    if (cached_occupancy(p, shape, mode, true) > 0) return true;
  }
  uint64_t row_bytes = 0;
  for (int c = 0; c < p.n_cols; ++c) row_bytes += (uint64_t)p.csize[c];
  int best_t = 0, best_s = 0;
  long best_score = -1;
  for (int t : {2048, 1024, 512, 256}) {
    for (int ns : {8, 6, 5, 4, 3, 2}) {
      if ((uint64_t)t * row_bytes > 48 * 1024) continue;
      set_stages(p, t, ns);
      const int occ = cached_occupancy(p, shape, mode, true);
      if (occ < 1) continue;
      const uint64_t inflight = (uint64_t)occ * ns * p.stage_bytes;
      const int warps = occ * (GB_BLOCK / 32);
      // enough bytes in flight per SM to cover HBM latency (~96 KB), then as
      // many resident warps as possible: the row loop is latency-bound
      const uint64_t capped = inflight < 96 * 1024 ? inflight : 96 * 1024;
      const long score = (long)(capped / 1024) * 100000L + (long)(warps > 48 ? 48 : warps) * 100 +
                         (long)(t / 256) * 2 - ns;
      if (score > best_score) {
        best_score = score;
        best_t = t;
        best_s = ns;
      }
    }
  }
  if (best_score < 0) return false;
  set_stages(p, best_t, best_s);
  return true;
}

// Launch the fused kernel, shrinking the per-CTA tables when they do not fit.
rel_status run_main(GbParams& p, int shape, int mode, cudaStream_t st) {
  const bool tma = tma_ok(p);
  for (;;) {
    if (configure_stages(p, shape, mode, tma)) return gb_launch_main(p, shape, mode, tma, st);
    if (p.tiny_frozen) {  // pinned placement cannot shrink: drop the layer
      mode = mode == MODE_TINY ? MODE_LAYERED : mode;
      p.tiny_frozen = 0;
      p.tiny_ns = 0;
      p.tiny_slots = 0;
      p.tiny_probes = 0;
    } else if (p.tiny_slots > 8) {
      p.tiny_slots >>= 1;
      p.tiny_probes = p.tiny_probes > p.tiny_slots ? p.tiny_slots : p.tiny_probes;
    } else if (p.tiny_slots) {
      p.tiny_slots = 0;
      p.tiny_probes = 0;
    } else if (p.smem_slots > 16) {
      p.smem_slots >>= 1;
    } else if (p.smem_slots && mode != MODE_KEYSET) {
      p.smem_slots = 0;
    } else {
      set_error("group-by: rows too wide to stage");
      return REL_E_UNSUPPORTED;
    }
  }
}

uint64_t gb_ws_bytes(int64_t slots, int32_t n_aggs) {
  return HEADER_BYTES + (uint64_t)slots * 8ull * (1ull + (uint64_t)n_aggs);
}

// ------------------------------------------------- partitioned variant (P)

constexpr uint32_t PART_MAX_GRID = 512;  // CTAs of the histogram / scatter passes

bool part_shape(int shape) {
  return shape == SHAPE_KV4_64 || shape == SHAPE_KV4_32 || shape == SHAPE_KV2_64 ||
         shape == SHAPE_KV2_32;
}

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Workspace after the header and spill table: histogram, partition starts,
// records.
struct PartLayout {
  uint64_t hist, starts, cursor, cursor1, l2_tiles, recs, recs1, end;
};

PartLayout part_layout(int64_t slots, int32_t n_aggs, int bits, int64_t n_rows) {
  PartLayout L;
  const uint64_t P = 1ull << bits;
  const uint64_t bins = 1ull << PART_L1_BITS;
  L.hist = align_up(gb_ws_bytes(slots, n_aggs), 256);
  L.starts = align_up(L.hist + 4ull * P * PART_MAX_GRID, 256);
  L.cursor = align_up(L.starts + 8ull * (P + 1), 256);
  L.cursor1 = align_up(L.cursor + 4ull * P, 256);
  L.l2_tiles = align_up(L.cursor1 + 4ull * bins, 256);
  L.recs = align_up(L.l2_tiles + 4ull * (bins + 1), 256);
  const uint64_t rec_bytes = sizeof(PartRec) * (uint64_t)(n_rows > 0 ? n_rows : 1);
  // level-1 records of the streaming scatter when there are two levels
  L.recs1 = align_up(L.recs + rec_bytes, 256);
  L.end = bits > PART_L1_BITS ? L.recs1 + rec_bytes : L.recs1;
  return L;
}

uint64_t plan_ws_bytes(const rel_plan* plan, int32_t n_aggs, int64_t n_rows) {
  if (plan->variant == REL_VAR_PARTITIONED)
    return part_layout(plan->slots, n_aggs, plan->part_bits, n_rows).end;
  return gb_ws_bytes(plan->slots, n_aggs);
}

// Histogram, scan, scatter, per-partition aggregation.  The histogram and
// scatter passes must see every row on the same CTA and classify it the same
// way, so both run with one grid size, one tile size and one pinned set.
rel_status run_partitioned(GbParams& p, const rel_plan* plan, int shape, const GbOut& o,
                           void* ws, cudaStream_t st) {
  const PartLayout L = part_layout(plan->slots, p.n_aggs, plan->part_bits, p.n_rows);
  uint8_t* base = (uint8_t*)ws;
  p.part_bits = (uint32_t)plan->part_bits;
  p.hist = (uint32_t*)(base + L.hist);
  p.part_start = (unsigned long long*)(base + L.starts);
  p.cursor = (unsigned int*)(base + L.cursor);
  p.cursor1 = (unsigned int*)(base + L.cursor1);
  p.l2_tiles = (unsigned int*)(base + L.l2_tiles);
  p.recs = (PartRec*)(base + L.recs);
  p.recs1 = p.part_bits > PART_L1_BITS ? (PartRec*)(base + L.recs1) : nullptr;
  uint32_t grid = 2u * (uint32_t)relhost::device_sms();
  p.fixed_grid = grid > PART_MAX_GRID ? PART_MAX_GRID : grid;
  const uint32_t agg_slots = p.smem_slots;
  p.smem_slots = 0;  // passes 1-2 keep only the pinned thread-private layer
  if (!p.tiny_frozen) {
    p.tiny_slots = 0;
    p.tiny_probes = 0;
  }
  rel_status r;
  if (!plan->tile_rows && gb_ppass_stream_eligible(p, shape, plan->n_hot)) {
    // the histogram's CTAs: as many as fit on the SMs at once
    p.fixed_grid = gb_ppass_stream_grid(p, shape, PART_MAX_GRID);
    if (p.fixed_grid < 1) return set_error("group-by: partition histogram does not fit"), REL_E_UNSUPPORTED;
    if ((r = gb_launch_ppass_stream(p, shape, false, st))) return r;
    if ((r = gb_launch_part_scan(p, false, st))) return r;
    if ((r = gb_launch_ppass_stream(p, shape, true, st))) return r;
    if (p.part_bits > PART_L1_BITS && (r = gb_launch_part_l2(p, st))) return r;
    p.smem_slots = agg_slots;
    return gb_launch_part_agg(p, shape, o, st);
  }
  const bool tma = tma_ok(p);
  if (!configure_stages(p, shape, MODE_PSCATTER, tma))
    return set_error("group-by: partition scatter does not fit"), REL_E_UNSUPPORTED;
  const int T = p.tile_rows, NS = p.n_stages;
  p.req_tile = T;
  p.req_stages = NS;
  if (!configure_stages(p, shape, MODE_PHIST, tma) || p.tile_rows != T)
    return set_error("group-by: partition histogram does not fit"), REL_E_UNSUPPORTED;
  if ((r = gb_launch_main(p, shape, MODE_PHIST, tma, st))) return r;
  if ((r = gb_launch_part_scan(p, true, st))) return r;
  set_stages(p, T, NS);
  if ((r = gb_launch_main(p, shape, MODE_PSCATTER, tma, st))) return r;
  p.smem_slots = agg_slots;
  return gb_launch_part_agg(p, shape, o, st);
}

// Many groups over key + value rows: partition instead of one big table.
void choose_partitioned(int64_t est, int64_t n_rows, rel_plan* plan) {
  uint64_t per = (uint64_t)(est / 768);
  int bits = 4;
  while (bits < PART_MAX_BITS && (1ull << bits) < per) ++bits;
  plan->variant = REL_VAR_PARTITIONED;
  plan->part_bits = bits;
  // each partition's table at load <= 0.5 on average (the partitions' key
  // counts vary by a few percent; a table that still fills spills its
  // partition to the global table)
  const uint64_t keys_per_part = (uint64_t)est >> bits;
  plan->smem_slots = (int32_t)next_pow2(keys_per_part * 2 < 256 ? 256 : keys_per_part * 2);
  if (plan->smem_slots > SHARED_MAX_SLOTS) plan->smem_slots = SHARED_MAX_SLOTS;
  plan->tiny_slots = 0;     // pinned heavy hitters only (from a sketch)
  // spill table: a partition whose keys do not all fit its table sends all
  // of them to the global table.  Sized for a quarter of the keys while the
  // partition tables stay below 0.4 load; for every key once they cannot
  // (more keys per partition than half a table of the largest size)
  uint64_t spill = (uint64_t)est / 4;
  if (2 * keys_per_part > (uint64_t)plan->smem_slots) spill = 2 * (uint64_t)est;
  plan->slots = (int64_t)next_pow2(spill > 65536 ? spill : 65536);
  (void)n_rows;
}

// Per-CTA layers for an expected number of groups.
void choose_layers(int64_t est, int words, rel_plan* plan) {
  plan->tiny_slots = 0;
  plan->smem_slots = 0;
  if (est <= 6 && words <= 6) {
    plan->variant = REL_VAR_SMEM;
    plan->tiny_slots = 8;
  } else if (est <= 12 && words <= 4) {
    plan->variant = REL_VAR_SMEM;
    plan->tiny_slots = 16;
  } else if (est <= 24 && words <= 2) {
    plan->variant = REL_VAR_SMEM;
    plan->tiny_slots = 32;
  } else if (est <= 2048) {
    plan->variant = REL_VAR_SMEM;
    plan->tiny_slots = words <= 6 ? 8 : 0;  // catches a skewed input's hottest keys
    plan->smem_slots = (int32_t)next_pow2((uint64_t)(2 * est));
  } else {
    plan->variant = REL_VAR_GLOBAL;
    plan->tiny_slots = words <= 6 ? 8 : 0;
    plan->smem_slots = 2048;
  }
}

constexpr uint32_t DEFAULT_TINY_MULT = 0x9E3779B1u;

// Host copy of the device's per-CTA slot hash (rel_internal.cuh, small_slot_of).
uint32_t host_small_slot(uint64_t ek, uint32_t mask, uint32_t mult) {
  const uint32_t f = (uint32_t)ek ^ (uint32_t)(ek >> 32);
  return (uint32_t)(((uint64_t)f * mult) >> 32) & mask;
}

// Place the hot keys at their hash slots; false on a collision.
bool place_hot(const int64_t* keys, int n, uint32_t slots, uint32_t mult, uint64_t* table) {
  for (uint32_t s = 0; s < slots; ++s) table[s] = 0;
  for (int i = 0; i < n; ++i) {
    const uint64_t ek = (uint64_t)keys[i] ^ KEY_FLIP;
    const uint32_t s = host_small_slot(ek, slots - 1, mult);
    if (table[s] != 0) return false;
    table[s] = ek;
  }
  return true;
}

// A multiplier that places every hot key in its own slot (0 if none found).
uint32_t perfect_mult(const int64_t* keys, int n, uint32_t slots) {
  uint64_t table[TINY_MAX_SLOTS];
  for (uint32_t i = 0; i < 4096; ++i) {
    const uint32_t mult = (DEFAULT_TINY_MULT + i * 0x3C6EF372u) | 1u;
    if (place_hot(keys, n, slots, mult, table)) return mult;
  }
  return 0;
}

// Thread-private slots a shape can afford (their shared memory grows with
// the aggregate words).
int32_t tiny_capacity(int words) {
  return words <= 2 ? 32 : words <= 4 ? 16 : words <= 6 ? 8 : 0;
}

// Pin the sample's frequent keys: all of them when the plan keeps every group
// thread-private, else the heavy hitters of a skewed sample.
void apply_sketch(const rel_sketch_info& s, int words, rel_plan* plan) {
  const int32_t cap = tiny_capacity(words);
  if (cap == 0 || s.kept == 0) return;
  int64_t top8 = 0;
  for (int i = 0; i < 8; ++i) top8 += s.top_count[i];
  const bool tiny_only = plan->tiny_slots && !plan->smem_slots;
  int want = 0;
  if (tiny_only) {
    want = s.ndv < plan->tiny_slots ? s.ndv : plan->tiny_slots;
  } else if (top8 * 20 >= (int64_t)s.kept) {  // top 8 keys hold >= 5 % of rows
    plan->tiny_slots = cap;
    for (int i = 0; i < REL_SKETCH_TOP && i < cap / 2; ++i)
      if (s.top_count[i] >= 2) want = i + 1;
  } else {
    plan->tiny_slots = 0;  // no heavy hitters: a thread-private layer only costs
    return;
  }
  int n = 0;
  for (int i = 0; i < want; ++i)
    if (s.top_key[i] != INT64_MIN) plan->hot_keys[n++] = s.top_key[i];
  if (n == 0) return;
  // the fewest slots with a collision-free placement: thread-private columns
  // cost shared memory that the staging ring needs for bytes in flight
  for (uint32_t slots = (uint32_t)next_pow2((uint64_t)(n < 2 ? 2 : n));
       slots <= (uint32_t)plan->tiny_slots; slots <<= 1) {
    const uint32_t mult = perfect_mult(plan->hot_keys, n, slots);
    if (mult) {
      plan->n_hot = n;
      plan->tiny_mult = mult;
      plan->tiny_slots = (int32_t)slots;
      return;
    }
  }
}

// Probe limits of the per-CTA layers: a layer that must hold every group
// scans it all; a cache in front of a larger layer gives up early.  Pinned
// hot keys sit at their own hash slot, so one probe decides.
rel_status set_layers(GbParams& p, const rel_plan* plan, int shape) {
  p.tiny_slots = (uint32_t)plan->tiny_slots;
  p.smem_slots = (uint32_t)plan->smem_slots;
  const bool tiny_only = p.tiny_slots && !p.smem_slots && plan->variant == REL_VAR_SMEM;
  p.tiny_probes = tiny_only ? p.tiny_slots : (p.tiny_slots ? 2u : 0u);
  p.shared_probes = plan->variant == REL_VAR_SMEM ? 16u : 4u;
  p.tiny_mult = plan->tiny_mult ? (plan->tiny_mult | 1u) : DEFAULT_TINY_MULT;
  p.tiny_frozen = 0;
  if (plan->n_hot > 0 && p.tiny_slots) {
    if (plan->n_hot > (int32_t)p.tiny_slots || plan->n_hot > REL_MAX_HOT ||
        !place_hot(plan->hot_keys, plan->n_hot, p.tiny_slots, p.tiny_mult, p.tiny_init))
      return set_error("group-by: the plan's hot keys collide under its multiplier"),
             REL_E_INVALID;
    p.tiny_frozen = 1;
    p.tiny_probes = 1;
    // at most four pinned keys, no CTA-shared layer, a shape of <= 5 words:
    // keep the accumulators in registers (dense ids in slot order).  With
    // more keys the register file costs more than it saves: 1e8 lineitem
    // rows with 6 pinned groups x 5 words take 1.49 ms in registers (132 of
    // them, one 9-warp CTA per SM) and 0.96 ms in thread-private shared words
    const bool regs_shape = shape == SHAPE_Q1 || shape == SHAPE_KV4_64 || shape == SHAPE_KV4_32 ||
                            shape == SHAPE_KV2_64 || shape == SHAPE_KV2_32;
    if (regs_shape && p.smem_slots == 0 && plan->n_hot <= 4 && p.tiny_slots <= 16) {
      p.tiny_ns = 4u;
      p.tiny_dense = 0;
      uint64_t j = 0;
      for (uint32_t s = 0; s < p.tiny_slots; ++s)
        if (p.tiny_init[s]) p.tiny_dense |= (j++) << (4 * s);
    }
  }
  return REL_OK;
}

// Kernel parameters of a sketch; returns the key width in bits.
int sketch_params(const rel_groupby_desc* d, SketchParams* sp) {
  std::memset(sp, 0, sizeof *sp);
  sp->n_rows = d->n_rows;
  for (int c = 0; c < d->n_cols; ++c) {
    sp->col[c] = (const uint8_t*)d->cols[c].data;
    sp->ctype[c] = d->cols[c].type;
  }
  sp->n_keys = d->n_keys;
  sp->n_preds = d->n_preds;
  int shift = 0, bits = 0;
  for (int k = d->n_keys - 1; k >= 0; --k) {
    const int w = elem_bits(d->cols[d->key_cols[k]].type);
    sp->key_col[k] = d->key_cols[k];
    sp->key_shift[k] = d->n_keys == 1 ? 0 : shift;
    sp->key_mask[k] = w >= 64 ? ~0ull : ((1ull << w) - 1);
    shift += w;
    bits += w;
  }
  for (int i = 0; i < d->n_preds; ++i) {
    sp->pred_col[i] = d->preds[i].col;
    sp->pred_lo[i] = d->preds[i].lo;
    sp->pred_hi[i] = d->preds[i].hi;
  }
  return bits;
}

// The host summary and the 264 features of a device sketch.
void sketch_fill(const rel_groupby_desc* d, const DevSketch& h, int bits, rel_sketch_info* out) {
  std::memset(out, 0, sizeof *out);
  out->n_rows = d->n_rows;
  out->sample_rows = h.sample_rows;
  out->kept = h.kept;
  out->ndv = h.ndv;
  out->singletons = h.singletons;
  out->runs = h.runs;
  out->key_bits = bits;
  out->key_min = h.key_min;
  out->key_max = h.key_max;
  for (int i = 0; i < REL_SKETCH_TOP; ++i) {
    out->top_key[i] = h.top_key[i];
    out->top_count[i] = h.top_count[i];
  }
  for (int i = 0; i < 256; ++i) {
    out->hll[i] = h.hll[i];
    out->features[i] = (float)(h.hll[i] / 57.0);
  }
  const double kept = h.kept, ndv = h.ndv;
  double top8 = 0;
  for (int i = 0; i < 8; ++i) top8 += h.top_count[i];
  float* f = out->features + 256;
  f[0] = (float)std::log2(d->n_rows > 1 ? (double)d->n_rows : 1.0);
  f[1] = (float)(h.kept ? ndv / kept : 0.0);
  f[2] = (float)(h.kept ? std::log2((double)((uint64_t)h.key_max - (uint64_t)h.key_min) + 1.0)
                        : 0.0);
  f[3] = (float)(h.kept ? h.top_count[0] / kept : 0.0);
  f[4] = (float)(h.kept ? top8 / kept : 0.0);
  f[5] = (float)(h.ndv ? h.singletons / ndv : 0.0);
  f[6] = (float)(h.runs ? kept / h.runs : 0.0);
  f[7] = (float)(bits / 64.0);
}

// The network REL_PLAN_LEARNED consults (caller-owned device memory).
const void* g_planner_bf16 = nullptr;
const float* g_planner_f32 = nullptr;

// slots of the exact pre-pass's first key set in the staged kernel (8 bytes
// each: 128 MB)
constexpr uint64_t EXACT_SET_L2_SLOTS = 1ull << 24;
// bytes of the streaming distinct count's first key set (and of each set of
// its hash-split passes): at this size a key's home bucket is almost always
// the only one probed, and the random bucket reads still mostly hit L2 while
// the column streams past
constexpr uint64_t EXACT_SET_FIRST_BYTES = 256ull << 20;
// entries of the streaming distinct count's per-CTA filter (0: none; the
// buckets of frequent keys are served by L1 instead)
constexpr uint32_t EXACT_FILTER_SLOTS = 0;

// Scratch after the sketch's: the 264 features and the 4 network outputs.
constexpr uint64_t LEARN_OUT_OFF = 1280;
constexpr uint64_t LEARN_HLL_OFF = 2048;  // full-data HyperLogLog registers
constexpr uint64_t LEARN_SCRATCH = LEARN_HLL_OFF + 4ull * HLL_REGS;
// the tail check: inputs of at least this many rows whose sample saw more
// than 3/4 of its distinct keys once are sized by a full-data HyperLogLog
constexpr int64_t LEARN_HLL_MIN_ROWS = 1ll << 22;
constexpr double LEARN_LOG2_MARGIN = 1.0;  // sizing headroom over the network's log2 estimate

// The learned sizing rule: from the network's outputs y (log2 of the group
// count, then the logits of the three variants) to an estimate and a
// variant.  Twice the predicted count plus 25 %: an underestimate costs a
// wasted run and the exact pre-pass, an overestimate only a larger table;
// never below the distinct keys already seen in the sample, never above the
// rows.  The variant is the most likely one among those allowed (ties go to
// the lower-numbered variant).
void learned_rule(const rel_sketch_info& info, const float* y, int64_t n_rows, bool p_ok,
                  int64_t* est, int* variant) {
  int64_t n = n_rows;
  if (std::isfinite(y[0])) {
    const double y0 = std::min(std::max((double)y[0], 0.0), 61.0) + LEARN_LOG2_MARGIN;
    const double g = std::ceil(std::exp2(y0) * 1.25);
    n = g < (double)n_rows ? (int64_t)g : n_rows;
  }
  if (n < info.ndv) n = info.ndv;
  *est = n;
  int best = REL_VAR_SMEM;
  for (int v = REL_VAR_GLOBAL; v <= REL_VAR_PARTITIONED; ++v)
    if ((v != REL_VAR_PARTITIONED || p_ok) && y[v] > y[best]) best = v;
  *variant = best;
}

// The learned sizing step: sketch, network forward, estimate and variant.
rel_status learned_estimate(const rel_groupby_desc* d, bool p_ok, void* ws, size_t ws_bytes,
                            rel_sketch_info* info, int64_t* est, int* variant, bool* hll_sized,
                            cudaStream_t st) {
  if (!g_planner_bf16) return set_error("plan: no planner network registered"), REL_E_INVALID;
  const uint64_t sk = rel_sketch_ws_bytes();
  rel_status r = rel_sketch(d, ws, ws_bytes, info, st);
  if (r) return r;
  float* dx = (float*)((uint8_t*)ws + sk);
  float* dy = (float*)((uint8_t*)ws + sk + LEARN_OUT_OFF);
  cudaError_t e = cudaMemcpyAsync(dx, info->features, sizeof info->features,
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemcpyAsync");
  if ((r = mlp_forward(g_planner_bf16, g_planner_f32, dx, 1, dy, nullptr, st))) return r;
  float y[REL_MLP_OUT];
  e = cudaMemcpyAsync(y, dy, sizeof y, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "reading the planner output");
  learned_rule(*info, y, d->n_rows, p_ok, est, variant);
  // A 4096-row sample says little about a long tail: when most keys it saw
  // occurred once and the input is large, one streaming pass of a full-data
  // HyperLogLog (about a fifth of the exact count's cost) sizes the table
  // instead -- standard error 1.6 %, sized with 25 % headroom -- and the
  // variant follows the rule by group count for that size.
  const bool stream_key = d->n_keys == 1 && d->n_preds == 0 &&
                          (d->cols[d->key_cols[0]].type == REL_I64 ||
                           d->cols[d->key_cols[0]].type == REL_I32);
  if (hll_sized) *hll_sized = false;
  if (stream_key && d->n_rows >= LEARN_HLL_MIN_ROWS && 4ll * info->singletons > 3ll * info->ndv) {
    uint32_t* dregs = (uint32_t*)((uint8_t*)ws + sk + LEARN_HLL_OFF);
    e = cudaMemsetAsync(dregs, 0, 4ull * HLL_REGS, st);
    if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
    rel_status r2 = hll_launch(d->cols[d->key_cols[0]].data, d->cols[d->key_cols[0]].type,
                               d->n_rows, dregs, st);
    if (r2) return r2;
    uint32_t regs[HLL_REGS];
    e = cudaMemcpyAsync(regs, dregs, sizeof regs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return relhost::cuda_fail(e, "reading the HyperLogLog registers");
    const double g = std::ceil(hll_estimate(regs) * 1.25);
    int64_t n = g < (double)d->n_rows ? (int64_t)g : d->n_rows;
    if (n < info->ndv) n = info->ndv;
    *est = n;
    *variant = 0;  // the rule by group count
    if (hll_sized) *hll_sized = true;
  }
  return REL_OK;
}

// Workspace of rel_plan_size_batched: the batched sketch's, then the feature
// rows, then the network outputs.
uint64_t batched_plan_feat_off(int32_t n) { return align_up(rel_sketch_batched_ws_bytes(n), 256); }
uint64_t batched_plan_out_off(int32_t n) {
  return batched_plan_feat_off(n) + align_up(4ull * REL_MLP_IN * (uint64_t)(n > 0 ? n : 1), 256);
}

// Table layers for a variant (0 = the rule by group count).
void choose_variant(int variant, int64_t est, int64_t n_rows, int words, bool p_ok,
                    rel_plan* plan) {
  switch (variant) {
    case REL_VAR_SMEM:
      choose_layers(est, words, plan);
      if (plan->variant != REL_VAR_SMEM) {
        plan->variant = REL_VAR_SMEM;
        plan->smem_slots = SHARED_MAX_SLOTS;
        plan->tiny_slots = words <= 6 ? 8 : 0;
      }
      break;
    case REL_VAR_GLOBAL:
      plan->variant = REL_VAR_GLOBAL;
      plan->tiny_slots = 0;
      plan->smem_slots = 0;
      break;
    case REL_VAR_PARTITIONED:
      choose_partitioned(est, n_rows, plan);
      break;
    default:
      choose_layers(est, words, plan);
      if (plan->variant == REL_VAR_GLOBAL && p_ok) choose_partitioned(est, n_rows, plan);
  }
}

// The exact distinct count of one int32 / int64 key column (no filter) in
// workspace ws of HEADER_BYTES + 8 * set_slots bytes.  First one pass with a
// key set of at most EXACT_SET_FIRST_BYTES (load <= ~0.5 up to 1.6e7 distinct
// keys; its random reads mostly hit L2); when the distinct keys overflow it,
// the whole workspace is split into K sets of at most EXACT_SET_FIRST_BYTES
// each (K <= 16) and K passes each count the keys of one hash range.  Every
// attempt gives the same count.
rel_status exact_distinct(const void* keys, int32_t key_type, int64_t n_rows, void* ws,
                          uint64_t set_slots, int64_t* est, cudaStream_t st) {
  DistinctParams dp;
  std::memset(&dp, 0, sizeof dp);
  dp.keys = keys;
  dp.n_rows = n_rows;
  dp.hdr = (WsHeader*)ws;
  dp.filter_slots = EXACT_FILTER_SLOTS;
  const uint64_t total_buckets = set_slots / DS_BUCKET_SLOTS;  // set_slots >= 16
  const uint64_t first_buckets = EXACT_SET_FIRST_BYTES / (8ull * DS_BUCKET_SLOTS);
  for (int attempt = 0; attempt < 2; ++attempt) {
    uint32_t passes = 1;
    uint64_t buckets = total_buckets < first_buckets ? total_buckets : first_buckets;
    if (attempt == 1) {
      if (total_buckets <= first_buckets) break;  // the first set was already the full one
      passes = (uint32_t)std::min<uint64_t>(16, (total_buckets + first_buckets - 1) / first_buckets);
      buckets = total_buckets / passes;
    }
    cudaError_t e = cudaMemsetAsync(ws, 0, HEADER_BYTES + 8ull * DS_BUCKET_SLOTS * buckets * passes, st);
    if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
    rel_status r;
    for (uint32_t k = 0; k < passes; ++k) {
      dp.n_pass = passes;
      dp.pass = k;
      dp.n_buckets = buckets;
      dp.set = (uint64_t*)((uint8_t*)ws + HEADER_BYTES) + (uint64_t)k * buckets * DS_BUCKET_SLOTS;
      if ((r = distinct_launch(dp, key_type, st))) return r;
    }
    HostHeader h;
    if ((r = read_header(ws, &h, st))) return r;
    if (h.overflow) continue;
    *est = (int64_t)h.aux + (h.n_side > 0 ? 1 : 0);
    return REL_OK;
  }
  return set_error("plan: key set overflow"), REL_E_OVERFLOW;
}

rel_status plan_groupby(const rel_groupby_desc* d, uint32_t flags, int64_t hint, void* ws,
                        size_t ws_bytes, rel_plan* plan, cudaStream_t st) {
  rel_status r = validate_desc(d);
  if (r) return r;
  std::memset(plan, 0, sizeof *plan);
  plan->flags = flags;
  GbParams p;
  Mapped m = match_shape(d, p);
  if (flags & REL_PLAN_GENERIC) m.shape = SHAPE_GENERIC;
  const bool p_ok = part_shape(m.shape) && d->n_rows < (1ll << 32);
  const int forced = (int)((flags & REL_PLAN_FORCE_MASK) >> 8);
  if (forced == REL_VAR_PARTITIONED && !p_ok)
    return set_error("plan: the partitioned variant needs one int32/int64 key, no filter, "
                     "one value column and fewer than 2^32 rows"),
           REL_E_UNSUPPORTED;
  rel_sketch_info info;
  bool have_info = false;
  int learned = 0;
  int64_t est;
  if (hint > 0) {
    est = hint;
  } else if ((flags & REL_PLAN_LEARNED) && !(flags & REL_PLAN_EXACT)) {
    plan->scratch_bytes = rel_sketch_ws_bytes() + LEARN_SCRATCH;
    if (!ws || ws_bytes < plan->scratch_bytes) {
      set_error("plan: learned sizing needs %llu workspace bytes",
                (unsigned long long)plan->scratch_bytes);
      return REL_E_CAPACITY;
    }
    if (d->n_rows == 0) {
      est = 0;
    } else {
      bool hll_sized = false;
      if ((r = learned_estimate(d, p_ok, ws, ws_bytes, &info, &est, &learned, &hll_sized, st)))
        return r;
      if (hll_sized) plan->flags |= REL_PLAN_HLL_SIZED;
      have_info = true;
    }
  } else if (flags & REL_PLAN_EXACT) {
    const uint64_t set_slots = next_pow2((uint64_t)(2 * d->n_rows < 16 ? 16 : 2 * d->n_rows));
    plan->scratch_bytes = HEADER_BYTES + 8ull * set_slots;
    if (!ws || ws_bytes < plan->scratch_bytes) {
      set_error("plan: exact sizing needs %llu workspace bytes",
                (unsigned long long)plan->scratch_bytes);
      return REL_E_CAPACITY;
    }
    if (d->n_rows == 0) {
      est = 0;
    } else {
      // reduced descriptor: the key and filter columns, one COUNT
      rel_col cols[REL_MAX_COLS];
      int32_t keys[REL_MAX_KEYS];
      rel_range_pred preds[REL_MAX_PREDS];
      int map[REL_MAX_COLS];
      for (int c = 0; c < REL_MAX_COLS; ++c) map[c] = -1;
      int nc = 0;
      auto use = [&](int c) {
        if (map[c] < 0) {
          map[c] = nc;
          cols[nc++] = d->cols[c];
        }
        return map[c];
      };
      for (int k = 0; k < d->n_keys; ++k) keys[k] = use(d->key_cols[k]);
      for (int i = 0; i < d->n_preds; ++i) {
        preds[i] = d->preds[i];
        preds[i].col = use(d->preds[i].col);
      }
      rel_agg cnt;
      std::memset(&cnt, 0, sizeof cnt);
      cnt.op = REL_COUNT;
      rel_groupby_desc kd = *d;
      kd.n_cols = nc;
      kd.cols = cols;
      kd.key_cols = keys;
      kd.preds = preds;
      kd.n_aggs = 1;
      kd.aggs = &cnt;
      GbParams kp;
      const int ident[REL_MAX_AGGS] = {0, 1, 2, 3, 4, 5, 6, 7};
      fill_params(&kd, ident, kp);
      // one int64 key and no filter: the specialised key/value reader, with
      // the key column standing in as the (unused) value column
      int kshape = SHAPE_GENERIC;
      if (m.shape != SHAPE_GENERIC && kd.n_keys == 1 && kd.n_preds == 0 &&
          kd.cols[keys[0]].type == REL_I64) {
        kshape = SHAPE_KVRT64;
        kp.r_a = keys[0];
      }
      kp.hdr = (WsHeader*)ws;
      kp.tkeys = (uint64_t*)((uint8_t*)ws + HEADER_BYTES);
      const int32_t kt = kd.cols[keys[0]].type;
      const bool stream_keys = !(flags & REL_PLAN_GENERIC) && kd.n_keys == 1 &&
                               kd.n_preds == 0 && (kt == REL_I64 || kt == REL_I32);
      if (stream_keys) {
        r = exact_distinct(kd.cols[keys[0]].data, kt, d->n_rows, ws, set_slots, &est, st);
        if (r) return r;
      } else {
        // First a key set of at most EXACT_SET_L2_SLOTS slots (128 MB: the
        // memset is small); only when the distinct keys overflow it, the full
        // 2 x rows set.  Both give the same count.
        uint64_t try_slots = set_slots < EXACT_SET_L2_SLOTS ? set_slots : EXACT_SET_L2_SLOTS;
        for (;;) {
          kp.log2_slots = log2_pow2(try_slots);
          kp.max_probe = (uint32_t)(try_slots < 4096 ? try_slots : 4096);
          kp.smem_slots = 2048;
          kp.shared_probes = 4;
          cudaError_t e = cudaMemsetAsync(ws, 0, HEADER_BYTES + 8ull * try_slots, st);
          if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
          if ((r = run_main(kp, kshape, MODE_KEYSET, st))) return r;
          HostHeader h;
          if ((r = read_header(ws, &h, st))) return r;
          if (h.timeout) return set_error("plan: a device wait timed out"), REL_E_TIMEOUT;
          if (h.overflow && try_slots < set_slots) {
            try_slots = set_slots;
            continue;
          }
          if (h.overflow) return set_error("plan: key set overflow"), REL_E_OVERFLOW;
          est = (int64_t)h.aux + (h.n_side > 0 ? 1 : 0);
          break;
        }
      }
    }
  } else {
    est = d->n_rows;
  }
  plan->est_groups = est;
  plan->slots = (int64_t)next_pow2((uint64_t)(2 * est < 16 ? 16 : 2 * est));
  choose_variant(forced ? forced : learned, est, d->n_rows, gb_shape_width(m.shape), p_ok, plan);
  plan->workspace_bytes = plan_ws_bytes(plan, d->n_aggs, d->n_rows);
  if ((flags & REL_PLAN_SKETCH) && d->n_rows > 0) {
    if (!have_info) {
      const uint64_t need = rel_sketch_ws_bytes();
      if (plan->scratch_bytes < need) plan->scratch_bytes = need;
      if (!ws || ws_bytes < plan->scratch_bytes) {
        set_error("plan: sketching needs %llu workspace bytes",
                  (unsigned long long)plan->scratch_bytes);
        return REL_E_CAPACITY;
      }
      if ((r = rel_sketch(d, ws, ws_bytes, &info, st))) return r;
    }
    apply_sketch(info, gb_shape_width(m.shape), plan);
  }
  return REL_OK;
}

// ------------------------------------------------------------------ join

struct JoinLayout {
  uint64_t slots;
  uint64_t bytes;
};

JoinLayout join_layout(int64_t n_build) {
  JoinLayout L;
  L.slots = next_pow2((uint64_t)(2 * n_build < 16 ? 16 : 2 * n_build));
  const uint64_t nb = (uint64_t)(n_build > 0 ? n_build : 1);
  L.bytes = HEADER_BYTES + L.slots * sizeof(JoinSlot) + align_up(nb * 8, 256) + nb * sizeof(JoinVal);
  return L;
}

JoinParams join_params(const rel_join_table* t) {
  JoinParams p;
  uint8_t* ws = (uint8_t*)t->ws;
  const uint64_t slots = (uint64_t)t->slots;
  p.hdr = (WsHeader*)ws;
  const uint64_t nb = (uint64_t)(t->n_build > 0 ? t->n_build : 1);
  p.slots = (JoinSlot*)(ws + HEADER_BYTES);
  p.pay = (long long*)(ws + HEADER_BYTES + sizeof(JoinSlot) * slots);
  p.side = (JoinVal*)((uint8_t*)p.pay + align_up(nb * 8, 256));
  p.log2_slots = t->log2_slots;
  return p;
}

rel_status validate_table(const rel_join_table* t) {
  if (!t || t->magic != TABLE_MAGIC || !t->ws || !is_pow2((uint64_t)t->slots))
    return set_error("join: not a built table"), REL_E_INVALID;
  return REL_OK;
}

rel_status count_pairs(const rel_join_probe_desc* pd, int64_t* out, cudaStream_t st) {
  if (!pd) return set_error("join: NULL probe descriptor"), REL_E_INVALID;
  rel_status r = validate_table(pd->table);
  if (r) return r;
  if (pd->n_probe < 0 || pd->n_probe > MAX_INDEX_ROWS)
    return set_error("join: n_probe outside [0, 2^31-1]"), REL_E_UNSUPPORTED;
  if (pd->n_probe > 0 && !pd->probe_keys) return set_error("join: no probe keys"), REL_E_INVALID;
  JoinParams p = join_params(pd->table);
  cudaError_t e = cudaMemsetAsync(&p.hdr->aux, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
  JoinOut o{nullptr, nullptr, nullptr, 0};
  if ((r = join_launch_probe(p, o, pd->probe_keys, pd->n_probe, false, st))) return r;
  HostHeader h;
  if ((r = read_header(p.hdr, &h, st))) return r;
  *out = (int64_t)h.aux;
  return REL_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

const char* rel_last_error(void) { return relhost::g_err; }

uint64_t rel_launch_count(void) { return relhost::g_launches.load(); }

int32_t rel_version(void) { return 100; }

void rel_profile_start(void) {
  relhost::g_prof.clear();
  relhost::g_pool_used = 0;
  relhost::g_prof_on = true;
}

int64_t rel_profile_stop(int32_t* ids, float* ms, int64_t max) {
  relhost::g_prof_on = false;
  int64_t n = 0;
  for (const auto& r : relhost::g_prof) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return -1;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return -1;
    if (n < max) {
      if (ids) ids[n] = r.id;
      if (ms) ms[n] = t;
    }
    ++n;
  }
  return n;
}

const char* rel_kernel_name(int32_t id) {
  static const char* names[] = {"gb_main_layered", "gb_main_keyset", "gb_compact",
                                "join_build", "join_probe", "join_count", "sketch", "gb_main_regs",
                                "gb_part_hist", "gb_part_scan", "gb_part_scatter",
                                "gb_part_agg", "mlp", "batch_a", "batch_b", "gb_stream", "hll",
                                "gb_part_l2"};
  return (id >= 0 && id < relhost::K_COUNT_IDS) ? names[id] : "?";
}

uint64_t rel_groupby_ws_bytes(int64_t slots, int32_t n_aggs) {
  if (slots < 0 || n_aggs < 0) return 0;
  return gb_ws_bytes(slots, n_aggs);
}

// ---------------------------------------------------------- planner network

rel_status rel_mlp_round(const float* params, void* bf16_params, void* stream) {
  if (!params || !bf16_params) return set_error("mlp: NULL parameters"), REL_E_INVALID;
  return mlp_round(params, bf16_params, as_stream(stream));
}

rel_status rel_mlp_forward(const void* bf16_params, const float* params, const float* x,
                           int32_t batch, float* out, float* acts, void* stream) {
  if (batch < 0) return set_error("mlp: batch < 0"), REL_E_INVALID;
  if (batch > 0 && (!bf16_params || !params || !x || !out))
    return set_error("mlp: NULL argument"), REL_E_INVALID;
  return mlp_forward(bf16_params, params, x, batch, out, acts, as_stream(stream));
}

uint64_t rel_mlp_ws_bytes(int32_t batch) {
  return batch < 0 ? 0 : sizeof(float) * (uint64_t)DZ_STRIDE * (uint64_t)(batch > 0 ? batch : 1);
}

rel_status rel_mlp_backward(const void* bf16_params, const float* x, const float* acts,
                            const float* out, const float* t_ndv, const int32_t* t_var,
                            int32_t batch, void* ws, size_t ws_bytes, float* grad, float* loss,
                            void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("mlp: workspace not 256-byte aligned"), REL_E_INVALID;
  if (batch < 0) return set_error("mlp: batch < 0"), REL_E_INVALID;
  if (!grad || !loss || (batch > 0 && (!bf16_params || !x || !acts || !out || !t_ndv || !t_var)))
    return set_error("mlp: NULL argument"), REL_E_INVALID;
  if (!ws || ws_bytes < rel_mlp_ws_bytes(batch))
    return set_error("mlp: workspace needs %llu bytes",
                     (unsigned long long)rel_mlp_ws_bytes(batch)),
           REL_E_CAPACITY;
  return mlp_backward(bf16_params, x, acts, out, t_ndv, t_var, batch, (float*)ws, grad, loss,
                      as_stream(stream));
}

rel_status rel_mlp_adamw(float* params, void* bf16_params, float* m, float* v, const float* grad,
                         int32_t step, float lr, float beta1, float beta2, float eps,
                         float weight_decay, void* stream) {
  if (!params || !bf16_params || !m || !v || !grad)
    return set_error("mlp: NULL argument"), REL_E_INVALID;
  if (step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return set_error("mlp: bad AdamW hyper-parameters"), REL_E_INVALID;
  MlpAdamW h;
  h.lr = lr;
  h.beta1 = beta1;
  h.beta2 = beta2;
  h.eps = eps;
  h.wd = weight_decay;
  h.bc1 = (float)(1.0 - std::pow((double)beta1, (double)step));
  h.bc2 = (float)(1.0 - std::pow((double)beta2, (double)step));
  return mlp_adamw(params, bf16_params, m, v, grad, h, as_stream(stream));
}

rel_status rel_planner_set(const void* bf16_params, const float* params) {
  if ((bf16_params == nullptr) != (params == nullptr))
    return set_error("planner: give both parameter copies or neither"), REL_E_INVALID;
  g_planner_bf16 = bf16_params;
  g_planner_f32 = params;
  return REL_OK;
}

uint64_t rel_plan_ws_bytes(const rel_plan* plan, int32_t n_aggs, int64_t n_rows) {
  if (!plan || n_aggs < 0 || n_rows < 0 || plan->slots < 0) return 0;
  if (plan->variant == REL_VAR_PARTITIONED &&
      (plan->part_bits < 0 || plan->part_bits > PART_MAX_BITS))
    return 0;
  return plan_ws_bytes(plan, n_aggs, n_rows);
}

uint64_t rel_sketch_ws_bytes(void) { return (sizeof(DevSketch) + 255) & ~(uint64_t)255; }

uint64_t rel_groupby_auto_ws_bytes(const rel_groupby_desc* d) {
  if (!d || d->n_rows < 0 || d->n_aggs < 0 || d->n_aggs > REL_MAX_AGGS) return 0;
  // every estimate is at most n_rows
  const uint64_t n = (uint64_t)d->n_rows;
  const uint64_t slots = next_pow2(2 * n < 16 ? 16 : 2 * n);
  const uint64_t p_slots = next_pow2(2 * n > 65536 ? 2 * n : 65536);
  uint64_t need = gb_ws_bytes((int64_t)slots, d->n_aggs);
  need = std::max(need, part_layout((int64_t)p_slots, d->n_aggs, PART_MAX_BITS, d->n_rows).end);
  need = std::max(need, HEADER_BYTES + 8 * slots);  // exact pre-pass key set
  need = std::max(need, rel_sketch_ws_bytes() + LEARN_SCRATCH);
  return need;
}

rel_status rel_groupby_auto(const rel_groupby_desc* d, uint32_t flags, void* ws, size_t ws_bytes,
                            int64_t* out_keys, int64_t* const* out_aggs, int64_t out_capacity,
                            int64_t* n_groups_host, rel_plan* plan_out, void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("group-by: workspace not 256-byte aligned"), REL_E_INVALID;
  rel_status r = validate_desc(d);
  if (r) return r;
  const uint64_t need = rel_groupby_auto_ws_bytes(d);
  if (!ws || ws_bytes < need)
    return set_error("group-by: workspace needs %llu bytes", (unsigned long long)need),
           REL_E_CAPACITY;
  cudaStream_t st = as_stream(stream);
  rel_plan plan;
  if ((r = plan_groupby(d, flags, 0, ws, ws_bytes, &plan, st))) return r;
  int64_t n = 0;
  r = rel_groupby_agg(d, &plan, ws, ws_bytes, out_keys, out_aggs, out_capacity, &n, stream);
  if (r == REL_E_OVERFLOW && !(plan.flags & REL_PLAN_EXACT)) {
    const uint32_t f2 =
        (flags & (REL_PLAN_SKETCH | REL_PLAN_GENERIC | REL_PLAN_FORCE_MASK)) | REL_PLAN_EXACT;
    if ((r = plan_groupby(d, f2, 0, ws, ws_bytes, &plan, st))) return r;
    plan.flags |= REL_PLAN_FELL_BACK;
    r = rel_groupby_agg(d, &plan, ws, ws_bytes, out_keys, out_aggs, out_capacity, &n, stream);
  }
  if (n_groups_host) *n_groups_host = n;
  if (plan_out) *plan_out = plan;
  return r;
}

rel_status rel_sketch(const rel_groupby_desc* d, void* ws, size_t ws_bytes, rel_sketch_info* out,
                      void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("sketch: workspace not 256-byte aligned"), REL_E_INVALID;
  rel_status r = validate_desc(d);
  if (r) return r;
  if (!out) return set_error("sketch: NULL output"), REL_E_INVALID;
  if (!ws || ws_bytes < rel_sketch_ws_bytes())
    return set_error("sketch: workspace needs %llu bytes",
                     (unsigned long long)rel_sketch_ws_bytes()),
           REL_E_CAPACITY;
  SketchParams sp;
  const int bits = sketch_params(d, &sp);
  cudaStream_t st = as_stream(stream);
  DevSketch* dev = (DevSketch*)ws;
  if ((r = sketch_launch(sp, dev, st))) return r;
  DevSketch h;
  cudaError_t e = cudaMemcpyAsync(&h, dev, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "reading the sketch");
  sketch_fill(d, h, bits, out);
  return REL_OK;
}

uint64_t rel_sketch_batched_ws_bytes(int32_t n) {
  if (n < 0) return 0;
  return align_up(sizeof(SketchParams) * (uint64_t)n, 256) +
         align_up(sizeof(DevSketch) * (uint64_t)n, 256) + 256;
}

rel_status rel_sketch_batched(const rel_groupby_desc* descs, int32_t n, void* ws, size_t ws_bytes,
                              rel_sketch_info* out, void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("sketch: workspace not 256-byte aligned"), REL_E_INVALID;
  if (n < 0 || (n > 0 && (!descs || !out)))
    return set_error("sketch: bad arguments"), REL_E_INVALID;
  if (n == 0) return REL_OK;
  rel_status r;
  for (int i = 0; i < n; ++i)
    if ((r = validate_desc(descs + i))) return r;
  if (!ws || ws_bytes < rel_sketch_batched_ws_bytes(n))
    return set_error("sketch: workspace needs %llu bytes",
                     (unsigned long long)rel_sketch_batched_ws_bytes(n)),
           REL_E_CAPACITY;
  std::vector<SketchParams> sp(n);
  std::vector<int> bits(n);
  for (int i = 0; i < n; ++i) bits[i] = sketch_params(descs + i, &sp[i]);
  uint8_t* base = (uint8_t*)align_up((uint64_t)(uintptr_t)ws, 256);
  SketchParams* dp = (SketchParams*)base;
  DevSketch* ds = (DevSketch*)(base + align_up(sizeof(SketchParams) * (uint64_t)n, 256));
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(dp, sp.data(), sizeof(SketchParams) * n, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemcpyAsync");
  if ((r = sketch_many_launch(dp, ds, n, st))) return r;
  std::vector<DevSketch> h(n);
  e = cudaMemcpyAsync(h.data(), ds, sizeof(DevSketch) * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "reading the sketches");
  for (int i = 0; i < n; ++i) sketch_fill(descs + i, h[i], bits[i], out + i);
  return REL_OK;
}

rel_status rel_plan_learned_rule(const rel_sketch_info* info, const float* y, int64_t n_rows,
                                 int32_t partitioned_ok, int64_t* est_groups, int32_t* variant) {
  if (!info || !y || !est_groups || !variant)
    return set_error("plan: NULL argument to the learned rule"), REL_E_INVALID;
  if (n_rows < 0) return set_error("plan: n_rows < 0"), REL_E_INVALID;
  int64_t est = 0;
  int v = REL_VAR_SMEM;
  learned_rule(*info, y, n_rows, partitioned_ok != 0, &est, &v);
  *est_groups = est;
  *variant = v;
  return REL_OK;
}

uint64_t rel_plan_size_batched_ws_bytes(int32_t n) {
  if (n < 0) return 0;
  return batched_plan_out_off(n) + align_up(4ull * REL_MLP_OUT * (uint64_t)(n > 0 ? n : 1), 256);
}

rel_status rel_plan_size_batched(const rel_groupby_desc* descs, int32_t n, uint32_t flags,
                                 void* ws, size_t ws_bytes, rel_plan* plans, void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("plan: workspace not 256-byte aligned"), REL_E_INVALID;
  if (n < 0 || (n > 0 && (!descs || !plans)))
    return set_error("plan: bad batched arguments"), REL_E_INVALID;
  if (!(flags & REL_PLAN_LEARNED) || (flags & (REL_PLAN_EXACT | REL_PLAN_GENERIC | REL_PLAN_FORCE_MASK)))
    return set_error("plan: batched planning is the learned form (REL_PLAN_LEARNED, optionally "
                     "REL_PLAN_SKETCH) only"),
           REL_E_UNSUPPORTED;
  if (n == 0) return REL_OK;
  rel_status r;
  for (int i = 0; i < n; ++i)
    if ((r = validate_desc(descs + i))) return r;
  if (!g_planner_bf16) return set_error("plan: no planner network registered"), REL_E_INVALID;
  const uint64_t need = rel_plan_size_batched_ws_bytes(n);
  if (!ws || ws_bytes < need)
    return set_error("plan: batched planning needs %llu workspace bytes", (unsigned long long)need),
           REL_E_CAPACITY;
  cudaStream_t st = as_stream(stream);
  std::vector<rel_sketch_info> info(n);
  if ((r = rel_sketch_batched(descs, n, ws, batched_plan_feat_off(n), info.data(), stream)))
    return r;
  std::vector<float> x((size_t)n * REL_MLP_IN), y((size_t)n * REL_MLP_OUT);
  for (int i = 0; i < n; ++i)
    std::memcpy(&x[(size_t)i * REL_MLP_IN], info[i].features, sizeof(float) * REL_MLP_IN);
  float* dx = (float*)((uint8_t*)ws + batched_plan_feat_off(n));
  float* dy = (float*)((uint8_t*)ws + batched_plan_out_off(n));
  cudaError_t e = cudaMemcpyAsync(dx, x.data(), sizeof(float) * x.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemcpyAsync");
  if ((r = mlp_forward(g_planner_bf16, g_planner_f32, dx, n, dy, nullptr, st))) return r;
  e = cudaMemcpyAsync(y.data(), dy, sizeof(float) * y.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "reading the planner outputs");
  for (int i = 0; i < n; ++i) {
    const rel_groupby_desc* d = descs + i;
    rel_plan* plan = plans + i;
    std::memset(plan, 0, sizeof *plan);
    plan->flags = flags;
    GbParams p;
    const Mapped m = match_shape(d, p);
    int64_t est = 0;
    int variant = REL_VAR_SMEM;
    // the batched launch has no partitioned variant
    learned_rule(info[i], &y[(size_t)i * REL_MLP_OUT], d->n_rows, false, &est, &variant);
    plan->est_groups = est;
    plan->slots = (int64_t)next_pow2((uint64_t)(2 * est < 16 ? 16 : 2 * est));
    choose_variant(variant, est, d->n_rows, gb_shape_width(m.shape), false, plan);
    plan->workspace_bytes = plan_ws_bytes(plan, d->n_aggs, d->n_rows);
    if (flags & REL_PLAN_SKETCH) apply_sketch(info[i], gb_shape_width(m.shape), plan);
  }
  return REL_OK;
}

uint64_t rel_key_hll_ws_bytes(void) { return 4ull * HLL_REGS; }

rel_status rel_key_hll(const void* keys, int32_t key_type, int64_t n, void* ws, size_t ws_bytes,
                       uint32_t* regs_host, double* estimate, void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("hll: workspace not 256-byte aligned"), REL_E_INVALID;
  if (n < 0 || (n > 0 && !keys) || !regs_host || !estimate)
    return set_error("hll: bad arguments"), REL_E_INVALID;
  if (key_type != REL_I32 && key_type != REL_I64)
    return set_error("hll: needs an int32 or int64 key"), REL_E_INVALID;
  if ((uintptr_t)keys % (key_type == REL_I64 ? 8 : 4))
    return set_error("hll: keys not aligned to their type"), REL_E_INVALID;
  if (!ws || ws_bytes < rel_key_hll_ws_bytes())
    return set_error("hll: workspace needs %llu bytes", (unsigned long long)rel_key_hll_ws_bytes()),
           REL_E_CAPACITY;
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaMemsetAsync(ws, 0, rel_key_hll_ws_bytes(), st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
  rel_status r = hll_launch(keys, key_type, n, (uint32_t*)ws, st);
  if (r) return r;
  e = cudaMemcpyAsync(regs_host, ws, rel_key_hll_ws_bytes(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "reading the HyperLogLog registers");
  *estimate = hll_estimate(regs_host);
  return REL_OK;
}

uint64_t rel_join_ws_bytes(int64_t n_build) {
  if (n_build < 0) return 0;
  return join_layout(n_build).bytes;
}

rel_status rel_plan_size(int32_t op, const void* desc, uint32_t flags, int64_t groups_hint,
                         void* ws, size_t ws_bytes, rel_plan* plan, void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("plan: workspace not 256-byte aligned"), REL_E_INVALID;
  if (!plan) return set_error("plan: NULL plan"), REL_E_INVALID;
  if (op == REL_OP_GROUPBY)
    return plan_groupby((const rel_groupby_desc*)desc, flags, groups_hint, ws, ws_bytes, plan,
                        as_stream(stream));
  if (op == REL_OP_JOIN_PROBE) {
    std::memset(plan, 0, sizeof *plan);
    plan->flags = flags;
    int64_t n = 0;
    rel_status r = count_pairs((const rel_join_probe_desc*)desc, &n, as_stream(stream));
    if (r) return r;
    plan->est_groups = n;
    return REL_OK;
  }
  set_error("plan: unknown op %d", op);
  return REL_E_INVALID;
}

rel_status rel_groupby_agg(const rel_groupby_desc* d, const rel_plan* plan, void* ws,
                           size_t ws_bytes, int64_t* out_keys, int64_t* const* out_aggs,
                           int64_t out_capacity, int64_t* n_groups_host, void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("group-by: workspace not 256-byte aligned"), REL_E_INVALID;
  rel_status r = validate_desc(d);
  if (r) return r;
  if (!plan) return set_error("group-by: NULL plan"), REL_E_INVALID;
  if (plan->slots < 16 || !is_pow2((uint64_t)plan->slots))
    return set_error("group-by: plan slots must be a power of two >= 16"), REL_E_INVALID;
  const int32_t ss = plan->smem_slots, ts = plan->tiny_slots;
  if (!(ss == 0 || (ss >= 16 && ss <= SHARED_MAX_SLOTS && is_pow2((uint64_t)ss))))
    return set_error("group-by: smem_slots must be 0 or a power of two in [16, 4096]"),
           REL_E_INVALID;
  if (!(ts == 0 || ts == 2 || ts == 4 || ts == 8 || ts == 16 || ts == 32))
    return set_error("group-by: tiny_slots must be 0, 2, 4, 8, 16 or 32"), REL_E_INVALID;
  const uint64_t need = gb_ws_bytes(plan->slots, d->n_aggs);  // zeroed part
  if (plan->variant == REL_VAR_PARTITIONED &&
      (plan->part_bits < 4 || plan->part_bits > PART_MAX_BITS || plan->smem_slots < 256 ||
       plan->smem_slots > SHARED_MAX_SLOTS || d->n_rows >= (1ll << 32)))
    return set_error("group-by: partitioned plans need part_bits in [4, 14], smem_slots in "
                     "[256, 4096] and fewer than 2^32 rows"),
           REL_E_INVALID;
  const uint64_t need_all = plan_ws_bytes(plan, d->n_aggs, d->n_rows);
  if (!ws || ws_bytes < need_all) {
    set_error("group-by: workspace needs %llu bytes", (unsigned long long)need_all);
    return REL_E_CAPACITY;
  }
  if (!ws || ws_bytes < need) {
    set_error("group-by: workspace needs %llu bytes", (unsigned long long)need);
    return REL_E_CAPACITY;
  }
  if (out_capacity < 0 || (out_capacity > 0 && (!out_keys || !out_aggs)))
    return set_error("group-by: bad outputs"), REL_E_INVALID;
  for (int a = 0; a < d->n_aggs; ++a)
    if (out_capacity > 0 && !out_aggs[a])
      return set_error("group-by: NULL aggregate output"), REL_E_INVALID;
  GbParams p;
  Mapped m = match_shape(d, p);
  if (plan->flags & REL_PLAN_GENERIC) {
    m.shape = SHAPE_GENERIC;
    for (int a = 0; a < REL_MAX_AGGS; ++a) m.perm[a] = a;
  }
  const GbParams roles = p;
  fill_params(d, m.perm, p);
  p.r_k0 = roles.r_k0;
  p.r_k1 = roles.r_k1;
  p.r_pred = roles.r_pred;
  p.r_a = roles.r_a;
  p.r_b = roles.r_b;
  p.r_d = roles.r_d;
  p.r_t = roles.r_t;
  GbOut o;
  std::memset(&o, 0, sizeof o);
  o.keys = out_keys;
  o.capacity = out_capacity;
  for (int a = 0; a < d->n_aggs; ++a) o.aggs[a] = out_capacity > 0 ? out_aggs[m.perm[a]] : nullptr;
  cudaStream_t st = as_stream(stream);
  p.hdr = (WsHeader*)ws;
  p.tkeys = (uint64_t*)((uint8_t*)ws + HEADER_BYTES);
  p.taggs = (unsigned long long*)(p.tkeys + plan->slots);
  p.log2_slots = log2_pow2((uint64_t)plan->slots);
  p.max_probe = (uint32_t)(plan->slots < 4096 ? plan->slots : 4096);
  if ((r = set_layers(p, plan, m.shape))) return r;
  p.wait_ns = WAIT_LIMIT_NS;
  if (plan->flags & REL_PLAN_TEST_STALL) {
    p.test_stall = 1;
    p.wait_ns = TEST_WAIT_LIMIT_NS;
  }
  if (plan->tile_rows || plan->n_stages) {
    const int32_t t = plan->tile_rows, ns = plan->n_stages;
    if (t < 256 || t > 4096 || !is_pow2((uint64_t)t) || ns < 2 || ns > GB_MAX_STAGES)
      return set_error("group-by: tile_rows must be a power of two in [256, 4096] and "
                       "n_stages in [2, 8]"),
             REL_E_INVALID;
    p.req_tile = t;
    p.req_stages = ns;
  }
  cudaError_t e = cudaMemsetAsync(ws, 0, need, st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
  if (plan->variant == REL_VAR_PARTITIONED && part_shape(m.shape)) {
    if ((r = run_partitioned(p, plan, m.shape, o, ws, st))) return r;
  } else if (!(plan->flags & REL_PLAN_GENERIC) && !plan->tile_rows &&
             gb_stream_eligible(p, m.shape, plan->n_hot)) {
    if ((r = gb_launch_stream(p, m.shape, st))) return r;
  } else {
    const int mode = p.tiny_ns ? MODE_TINY : MODE_LAYERED;
    if ((r = run_main(p, m.shape, mode, st))) return r;
  }
  if ((r = gb_launch_compact(p, o, st))) return r;
  if (!n_groups_host) return REL_OK;
  HostHeader h;
  if ((r = read_header(ws, &h, st))) return r;
  *n_groups_host = (int64_t)h.n_out;
  if (h.timeout & 2u)  // a partition pass found a count it did not expect; nothing was written past
    return set_error("group-by: the partition passes disagreed on a partition's size"), REL_E_CUDA;
  if (h.timeout) return set_error("group-by: a device wait timed out"), REL_E_TIMEOUT;
  if (h.overflow) {
    *n_groups_host = -1;
    return set_error("group-by: more groups than the plan's %lld slots hold",
                     (long long)plan->slots),
           REL_E_OVERFLOW;
  }
  if ((int64_t)h.n_out > out_capacity)
    return set_error("group-by: %llu groups exceed the output capacity", h.n_out), REL_E_CAPACITY;
  return REL_OK;
}

rel_status rel_join_build(const int64_t* keys, const int64_t* payload, int64_t n_build, void* ws,
                          size_t ws_bytes, rel_join_table* table, void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("join: workspace not 256-byte aligned"), REL_E_INVALID;
  if (!table) return set_error("join: NULL table handle"), REL_E_INVALID;
  if (n_build < 0 || n_build > MAX_INDEX_ROWS)
    return set_error("join: n_build outside [0, 2^31-1]"), REL_E_UNSUPPORTED;
  if (n_build > 0 && (!keys || !payload)) return set_error("join: no build columns"), REL_E_INVALID;
  const JoinLayout L = join_layout(n_build);
  if (!ws || ws_bytes < L.bytes) {
    set_error("join: workspace needs %llu bytes", (unsigned long long)L.bytes);
    return REL_E_CAPACITY;
  }
  std::memset(table, 0, sizeof *table);
  table->ws = ws;
  table->slots = (int64_t)L.slots;
  table->n_build = n_build;
  table->log2_slots = log2_pow2(L.slots);
  table->magic = TABLE_MAGIC;
  cudaStream_t st = as_stream(stream);
  cudaError_t e = cudaMemsetAsync(ws, 0, HEADER_BYTES + sizeof(JoinSlot) * L.slots, st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
  return join_launch_build(join_params(table), keys, payload, n_build, st);
}

rel_status rel_join_probe(const rel_join_table* t, const int64_t* probe_keys, int64_t n_probe,
                          int32_t* out_probe_idx, int32_t* out_build_idx, int64_t* out_payload,
                          int64_t out_capacity, int64_t* n_pairs_host, void* stream) {
  rel_status r = validate_table(t);
  if (r) return r;
  if (n_probe < 0 || n_probe > MAX_INDEX_ROWS)
    return set_error("join: n_probe outside [0, 2^31-1]"), REL_E_UNSUPPORTED;
  if (n_probe > 0 && !probe_keys) return set_error("join: no probe keys"), REL_E_INVALID;
  if (out_capacity < 0 ||
      (out_capacity > 0 && (!out_probe_idx || !out_build_idx || !out_payload)))
    return set_error("join: bad outputs"), REL_E_INVALID;
  cudaStream_t st = as_stream(stream);
  JoinParams p = join_params(t);
  cudaError_t e = cudaMemsetAsync(&p.hdr->n_out, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
  JoinOut o{out_probe_idx, out_build_idx, out_payload, out_capacity};
  if ((r = join_launch_probe(p, o, probe_keys, n_probe, true, st))) return r;
  if (!n_pairs_host) return REL_OK;
  HostHeader h;
  if ((r = read_header(p.hdr, &h, st))) return r;
  *n_pairs_host = (int64_t)h.n_out;
  if (h.overflow) return set_error("join: build table overflow"), REL_E_OVERFLOW;
  if ((int64_t)h.n_out > out_capacity)
    return set_error("join: %llu pairs exceed the output capacity", h.n_out), REL_E_CAPACITY;
  return REL_OK;
}

}  // extern "C"
