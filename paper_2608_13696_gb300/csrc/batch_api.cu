// C ABI of the batched execution mode (include/rel.h, "batched execution"):
// layout of the workspace, descriptor upload, run, results and the
// autotuner over tile shape, probe width and shared-memory placement.
#include <algorithm>
#include <cstring>
#include <vector>

#include "batch.cuh"

using namespace rel;
using relhost::set_error;

namespace {

constexpr uint64_t BATCH_MAGIC = 0x52454c4241544348ull;  // "RELBATCH"

struct HandleImpl {
  uint64_t magic;
  uint8_t* ws;
  int32_t n_g, n_j;
  int32_t block, items, width, smem_bytes;
  int32_t grid_a, grid_b;
  uint64_t zero_off, zero_bytes;
  uint64_t off_gb, off_jn, off_gbt, off_jbt, off_jpt, off_gct, off_ctr, off_gst, off_jst;
};
static_assert(sizeof(HandleImpl) <= sizeof(rel_batch_handle), "handle fits");

uint64_t align256(uint64_t x) { return (x + 255) & ~(uint64_t)255; }

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

int log2u(uint64_t x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

uint64_t join_slots(int64_t n_build) {
  return next_pow2((uint64_t)(2 * n_build < 16 ? 16 : 2 * n_build));
}

int32_t smem_slots_for(const rel_batch_groupby& g, const rel_batch_config& c) {
  if (c.smem_max_groups <= 0 || g.est_groups > c.smem_max_groups) return 0;
  const uint64_t s = next_pow2((uint64_t)(2 * g.est_groups < 16 ? 16 : 2 * g.est_groups));
  return (int32_t)std::min<uint64_t>(s, BATCH_MAX_SMEM_SLOTS);
}

struct Layout {
  uint64_t off_gb, off_jn, off_gbt, off_jbt, off_jpt, off_gct, off_ctr, off_gst, off_jst;
  std::vector<uint64_t> gtab, jtab, jside;  // table (and side list) offsets
  uint64_t zero_end, total;
};

Layout layout(const rel_batch_groupby* gb, int n_g, const rel_batch_join* jn, int n_j) {
  Layout L;
  uint64_t o = 256;
  L.off_gb = o;
  o = align256(o + sizeof(BatchGb) * (uint64_t)n_g);
  L.off_jn = o;
  o = align256(o + sizeof(BatchJoin) * (uint64_t)n_j);
  L.off_gbt = o;
  o = align256(o + 8ull * (n_g + 1));
  L.off_jbt = o;
  o = align256(o + 8ull * (n_j + 1));
  L.off_jpt = o;
  o = align256(o + 8ull * (n_j + 1));
  L.off_gct = o;
  o = align256(o + 8ull * (n_g + 1));
  // zeroed before every run: counters, statuses, tables
  L.off_ctr = o;
  o = align256(o + 16);
  L.off_gst = o;
  o = align256(o + sizeof(BatchStatus) * (uint64_t)n_g);
  L.off_jst = o;
  o = align256(o + sizeof(BatchStatus) * (uint64_t)n_j);
  L.gtab.resize(n_g);
  for (int i = 0; i < n_g; ++i) {
    L.gtab[i] = o;
    o = align256(o + (uint64_t)gb[i].slots * 8ull * (1ull + (uint64_t)gb[i].n_aggs));
  }
  L.jtab.resize(n_j);
  for (int i = 0; i < n_j; ++i) {
    L.jtab[i] = o;
    o = align256(o + join_slots(jn[i].n_build) * (8 + sizeof(JoinVal)));
  }
  L.zero_end = o;
  L.jside.resize(n_j);
  for (int i = 0; i < n_j; ++i) {
    L.jside[i] = o;
    o = align256(o + sizeof(JoinVal) * (uint64_t)std::max<int64_t>(1, jn[i].n_build));
  }
  L.total = o;
  return L;
}

rel_status validate(const rel_batch_groupby* gb, int32_t n_g, const rel_batch_join* jn,
                    int32_t n_j) {
  if (n_g < 0 || n_j < 0 || (n_g && !gb) || (n_j && !jn))
    return set_error("batch: bad instance arrays"), REL_E_INVALID;
  for (int i = 0; i < n_g; ++i) {
    const rel_batch_groupby& g = gb[i];
    if (g.key_type != REL_I32 && g.key_type != REL_I64)
      return set_error("batch: group-by %d: key_type must be REL_I32 or REL_I64", i), REL_E_INVALID;
    if (g.n_aggs < 1 || g.n_aggs > REL_BATCH_MAX_AGGS)
      return set_error("batch: group-by %d: n_aggs must be 1..4", i), REL_E_INVALID;
    bool all_count = true;
    for (int a = 0; a < g.n_aggs; ++a) {
      if (g.ops[a] < REL_SUM || g.ops[a] > REL_MAX)
        return set_error("batch: group-by %d: bad aggregate op", i), REL_E_INVALID;
      all_count &= g.ops[a] == REL_COUNT;
    }
    if (g.n_rows < 0 || (g.n_rows > 0 && (!g.keys || (!g.vals && !all_count))))
      return set_error("batch: group-by %d: bad input columns", i), REL_E_INVALID;
    if (g.slots < 16 || !is_pow2((uint64_t)g.slots) || g.slots > (1ll << 40))
      return set_error("batch: group-by %d: slots must be a power of two in [16, 2^40]", i),
             REL_E_INVALID;
    if (g.est_groups < 0 || g.out_capacity < 0)
      return set_error("batch: group-by %d: negative size", i), REL_E_INVALID;
    if (g.out_capacity > 0) {
      if (!g.out_keys) return set_error("batch: group-by %d: NULL output", i), REL_E_INVALID;
      for (int a = 0; a < g.n_aggs; ++a)
        if (!g.out_aggs[a]) return set_error("batch: group-by %d: NULL output", i), REL_E_INVALID;
    }
  }
  for (int i = 0; i < n_j; ++i) {
    const rel_batch_join& j = jn[i];
    if (j.n_build < 0 || j.n_probe < 0 || j.out_capacity < 0)
      return set_error("batch: join %d: negative size", i), REL_E_INVALID;
    if (j.n_build >= (1ll << 31) || j.n_probe >= (1ll << 31))
      return set_error("batch: join %d: sides must have fewer than 2^31 rows", i),
             REL_E_UNSUPPORTED;
    if ((j.n_build > 0 && (!j.build_keys || !j.build_payload)) || (j.n_probe > 0 && !j.probe_keys))
      return set_error("batch: join %d: bad input columns", i), REL_E_INVALID;
    if (j.out_capacity > 0 && (!j.out_probe_idx || !j.out_build_idx || !j.out_payload))
      return set_error("batch: join %d: NULL output", i), REL_E_INVALID;
  }
  return REL_OK;
}

rel_status validate_config(const rel_batch_config* c) {
  if (!c) return set_error("batch: NULL config"), REL_E_INVALID;
  if (c->block != 128 && c->block != 256 && c->block != 512)
    return set_error("batch: block must be 128, 256 or 512"), REL_E_INVALID;
  if (c->items != 4 && c->items != 8 && c->items != 16)
    return set_error("batch: items must be 4, 8 or 16"), REL_E_INVALID;
  if (c->probe_width != 1 && c->probe_width != 2 && c->probe_width != 4 && c->probe_width != 8)
    return set_error("batch: probe_width must be 1, 2, 4 or 8"), REL_E_INVALID;
  if (c->smem_max_groups < 0 || c->smem_max_groups > BATCH_MAX_SMEM_SLOTS / 2)
    return set_error("batch: smem_max_groups must be in [0, %d]", BATCH_MAX_SMEM_SLOTS / 2),
           REL_E_INVALID;
  return REL_OK;
}

BatchArgs args_of(const HandleImpl& h) {
  BatchArgs a;
  a.gb = (const BatchGb*)(h.ws + h.off_gb);
  a.jn = (const BatchJoin*)(h.ws + h.off_jn);
  a.gb_tiles = (const long long*)(h.ws + h.off_gbt);
  a.jb_tiles = (const long long*)(h.ws + h.off_jbt);
  a.jp_tiles = (const long long*)(h.ws + h.off_jpt);
  a.gc_tiles = (const long long*)(h.ws + h.off_gct);
  a.gst = (BatchStatus*)(h.ws + h.off_gst);
  a.jst = (BatchStatus*)(h.ws + h.off_jst);
  a.ctr = (unsigned long long*)(h.ws + h.off_ctr);
  a.n_g = h.n_g;
  a.n_j = h.n_j;
  return a;
}

rel_status prepare(const rel_batch_groupby* gb, int32_t n_g, const rel_batch_join* jn, int32_t n_j,
                   const rel_batch_config* cfg, void* ws, size_t ws_bytes, HandleImpl* h,
                   cudaStream_t st) {
  rel_status r = validate(gb, n_g, jn, n_j);
  if (r) return r;
  if ((r = validate_config(cfg))) return r;
  const Layout L = layout(gb, n_g, jn, n_j);
  if (!ws || ws_bytes < L.total)
    return set_error("batch: workspace needs %llu bytes", (unsigned long long)L.total),
           REL_E_CAPACITY;
  uint8_t* base = (uint8_t*)ws;
  const long long T = (long long)cfg->block * cfg->items;
  // host image of the descriptor region [off_gb, off_ctr)
  std::vector<uint8_t> img(L.off_ctr - L.off_gb, 0);
  auto at = [&](uint64_t off) { return img.data() + (off - L.off_gb); };
  int smem_bytes = 0;
  long long* gbt = (long long*)at(L.off_gbt);
  long long* gct = (long long*)at(L.off_gct);
  gbt[0] = gct[0] = 0;
  for (int i = 0; i < n_g; ++i) {
    const rel_batch_groupby& g = gb[i];
    BatchGb d;
    std::memset(&d, 0, sizeof d);
    d.keys = g.keys;
    d.vals = g.vals;
    d.n_rows = g.n_rows;
    d.tkeys = (uint64_t*)(base + L.gtab[i]);
    d.taggs = (unsigned long long*)(d.tkeys + g.slots);
    d.out_keys = g.out_keys;
    for (int a = 0; a < g.n_aggs; ++a) {
      d.out_aggs[a] = g.out_aggs[a];
      d.ops[a] = g.ops[a];
    }
    d.out_capacity = g.out_capacity;
    d.key_type = g.key_type;
    d.n_aggs = g.n_aggs;
    d.log2_slots = log2u((uint64_t)g.slots);
    d.smem_slots = smem_slots_for(g, *cfg);
    d.max_probe = (uint32_t)std::min<int64_t>(g.slots, 4096);
    d.span = BATCH_GB_SPAN;
    smem_bytes = std::max(smem_bytes, d.smem_slots * 8 * (1 + g.n_aggs));
    std::memcpy(at(L.off_gb) + sizeof(BatchGb) * i, &d, sizeof d);
    gbt[i + 1] = gbt[i] + (g.n_rows + T * BATCH_GB_SPAN - 1) / (T * BATCH_GB_SPAN);
    gct[i + 1] = gct[i] + (g.slots + T - 1) / T;
  }
  long long* jbt = (long long*)at(L.off_jbt);
  long long* jpt = (long long*)at(L.off_jpt);
  jbt[0] = jpt[0] = 0;
  for (int i = 0; i < n_j; ++i) {
    const rel_batch_join& j = jn[i];
    const uint64_t slots = join_slots(j.n_build);
    BatchJoin d;
    std::memset(&d, 0, sizeof d);
    d.bkeys = j.build_keys;
    d.bpay = j.build_payload;
    d.n_build = j.n_build;
    d.pkeys = j.probe_keys;
    d.n_probe = j.n_probe;
    d.tkeys = (uint64_t*)(base + L.jtab[i]);
    d.tvals = (JoinVal*)(d.tkeys + slots);
    d.side = (JoinVal*)(base + L.jside[i]);
    d.o_pi = j.out_probe_idx;
    d.o_bi = j.out_build_idx;
    d.o_pay = j.out_payload;
    d.capacity = j.out_capacity;
    d.log2_slots = log2u(slots);
    d.max_probe = (uint32_t)std::min<uint64_t>(slots, 4096);
    std::memcpy(at(L.off_jn) + sizeof(BatchJoin) * i, &d, sizeof d);
    jbt[i + 1] = jbt[i] + (j.n_build + T - 1) / T;
    jpt[i + 1] = jpt[i] + (j.n_probe + T - 1) / T;
  }
  cudaError_t e = cudaMemcpyAsync(base + L.off_gb, img.data(), img.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "uploading the batch");
  int pa = 0, pb = 0;
  if ((r = batch_occupancy(cfg->block, cfg->items, cfg->probe_width, smem_bytes, &pa, &pb)))
    return r;
  if (pa < 1 || pb < 1)
    return set_error("batch: config does not fit on an SM"), REL_E_UNSUPPORTED;
  const long long items_a = (n_j ? jbt[n_j] : 0) + (n_g ? gbt[n_g] : 0);
  const long long items_b = (n_j ? jpt[n_j] : 0) + (n_g ? gct[n_g] : 0);
  const long long sms = relhost::device_sms();
  std::memset(h, 0, sizeof *h);
  h->magic = BATCH_MAGIC;
  h->ws = base;
  h->n_g = n_g;
  h->n_j = n_j;
  h->block = cfg->block;
  h->items = cfg->items;
  h->width = cfg->probe_width;
  h->smem_bytes = smem_bytes;
  h->grid_a = (int32_t)std::max(1ll, std::min(items_a, sms * pa));
  h->grid_b = (int32_t)std::max(1ll, std::min(items_b, sms * pb));
  h->zero_off = L.off_ctr;
  h->zero_bytes = L.zero_end - L.off_ctr;
  h->off_gb = L.off_gb;
  h->off_jn = L.off_jn;
  h->off_gbt = L.off_gbt;
  h->off_jbt = L.off_jbt;
  h->off_jpt = L.off_jpt;
  h->off_gct = L.off_gct;
  h->off_ctr = L.off_ctr;
  h->off_gst = L.off_gst;
  h->off_jst = L.off_jst;
  return REL_OK;
}

rel_status run(const HandleImpl& h, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(h.ws + h.zero_off, 0, h.zero_bytes, st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
  return batch_launch(args_of(h), h.block, h.items, h.width, h.smem_bytes, h.grid_a, h.grid_b, st);
}

const HandleImpl* impl(const rel_batch_handle* h) {
  const HandleImpl* p = (const HandleImpl*)h;
  return (p && p->magic == BATCH_MAGIC) ? p : nullptr;
}

}  // namespace

extern "C" {

uint64_t rel_batch_ws_bytes(const rel_batch_groupby* gb, int32_t n_gb, const rel_batch_join* jn,
                            int32_t n_jn) {
  if (validate(gb, n_gb, jn, n_jn)) return 0;
  return layout(gb, n_gb, jn, n_jn).total;
}

rel_status rel_batch_prepare(const rel_batch_groupby* gb, int32_t n_gb, const rel_batch_join* jn,
                             int32_t n_jn, const rel_batch_config* cfg, void* ws, size_t ws_bytes,
                             rel_batch_handle* handle, void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("batch: workspace not 256-byte aligned"), REL_E_INVALID;
  if (!handle) return set_error("batch: NULL handle"), REL_E_INVALID;
  return prepare(gb, n_gb, jn, n_jn, cfg, ws, ws_bytes, (HandleImpl*)handle, (cudaStream_t)stream);
}

rel_status rel_batch_run(const rel_batch_handle* handle, void* stream) {
  const HandleImpl* h = impl(handle);
  if (!h) return set_error("batch: not a prepared handle"), REL_E_INVALID;
  return run(*h, (cudaStream_t)stream);
}

rel_status rel_batch_results(const rel_batch_handle* handle, int64_t* n_out, uint32_t* flags,
                             void* stream) {
  const HandleImpl* h = impl(handle);
  if (!h) return set_error("batch: not a prepared handle"), REL_E_INVALID;
  const int n = h->n_g + h->n_j;
  if (n == 0) return REL_OK;
  if (!n_out || !flags) return set_error("batch: NULL result arrays"), REL_E_INVALID;
  std::vector<BatchStatus> sg(h->n_g), sj(h->n_j);
  std::vector<BatchGb> dg(h->n_g);
  std::vector<BatchJoin> dj(h->n_j);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (h->n_g) {
    e = cudaMemcpyAsync(sg.data(), h->ws + h->off_gst, sizeof(BatchStatus) * h->n_g,
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dg.data(), h->ws + h->off_gb, sizeof(BatchGb) * h->n_g,
                          cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess && h->n_j) {
    e = cudaMemcpyAsync(sj.data(), h->ws + h->off_jst, sizeof(BatchStatus) * h->n_j,
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dj.data(), h->ws + h->off_jn, sizeof(BatchJoin) * h->n_j,
                          cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "reading batch results");
  for (int i = 0; i < h->n_g; ++i) {
    n_out[i] = (int64_t)sg[i].n_out;
    flags[i] = (sg[i].overflow ? 1u : 0u) | ((int64_t)sg[i].n_out > dg[i].out_capacity ? 2u : 0u);
  }
  for (int i = 0; i < h->n_j; ++i) {
    n_out[h->n_g + i] = (int64_t)sj[i].n_out;
    flags[h->n_g + i] =
        (sj[i].overflow ? 1u : 0u) | ((int64_t)sj[i].n_out > dj[i].capacity ? 2u : 0u);
  }
  return REL_OK;
}

rel_status rel_batch_autotune(const rel_batch_groupby* gb, int32_t n_gb, const rel_batch_join* jn,
                              int32_t n_jn, const rel_batch_config* cands, int32_t n_cands,
                              int32_t reps, void* ws, size_t ws_bytes, rel_batch_handle* handle,
                              rel_batch_config* best, float* ms, void* stream) {
  if (relhost::ws_unaligned(ws))
    return set_error("batch: workspace not 256-byte aligned"), REL_E_INVALID;
  if (!cands || n_cands < 1 || reps < 1 || !handle || !best)
    return set_error("batch: bad autotune arguments"), REL_E_INVALID;
  rel_status r = validate(gb, n_gb, jn, n_jn);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_error("batch: cudaEventCreate failed"), REL_E_CUDA;
  int best_i = -1;
  float best_ms = 0.f;
  std::vector<float> t(reps);
  for (int c = 0; c < n_cands && r == REL_OK; ++c) {
    if (ms) ms[c] = -1.f;
    HandleImpl h;
    const rel_status rc = prepare(gb, n_gb, jn, n_jn, cands + c, ws, ws_bytes, &h, st);
    if (rc == REL_E_INVALID || rc == REL_E_UNSUPPORTED) continue;  // not a usable config
    if (rc) {
      r = rc;
      break;
    }
    if ((r = run(h, st))) break;
    for (int k = 0; k < reps && r == REL_OK; ++k) {
      cudaEventRecord(e0, st);
      r = run(h, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) r = relhost::cuda_fail(cudaGetLastError(), "autotune");
      cudaEventElapsedTime(&t[k], e0, e1);
    }
    if (r) break;
    std::sort(t.begin(), t.end());
    const float med = t[reps / 2];
    if (ms) ms[c] = med;
    if (best_i < 0 || med < best_ms) {
      best_i = c;
      best_ms = med;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r) return r;
  if (best_i < 0) return set_error("batch: no candidate config is usable"), REL_E_INVALID;
  *best = cands[best_i];
  return prepare(gb, n_gb, jn, n_jn, best, ws, ws_bytes, (HandleImpl*)handle, st);
}

}  // extern "C"
