// ORACLE -- test infrastructure, not the product.
//
// A plain, single-threaded CPU statement of what the relational hot path
// computes.  Only the tests, the smoke check and the CPU-baseline leg of the
// benchmark load it; the library under paper_2608_13696_gb300/ never does.
// It shares no source with the CUDA path: no headers, hash functions, table
// layouts or constants.
//
// The paper (a measurement study of GPU relational operators) defines the
// operators by what they produce, not by a kernel design:
//   * group-by aggregation, fused with a filter and projected expressions
//     (Sec. 2.3 operator API; Sec. 7, Table 9: single_pass_shmem_aggs_kernel,
//     compute_column_kernel, transform_kernel);
//   * hash equi-join: build, count of matches, materialisation of matching
//     pairs with a payload gather  out[i] = in[map[i]]  (Sec. 7: insert_if_n,
//     count, retrieve, transform_kernel).
// Each function below is that plain definition written out:
//   group-by  -> one std::unordered_map entry per distinct key, rows visited
//                in order, then sorted by key;
//   join      -> nested loops on small inputs, std::unordered_multimap on
//                larger ones, pairs sorted by (probe row, build row).
// All aggregate arithmetic is exact two's-complement int64 (wrap mod 2^64);
// the paper's workloads are integer and fixed point (Sec. 5, Table 5).

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace {

enum { T_U8 = 0, T_I32 = 1, T_I64 = 2 };
enum { A_SUM = 0, A_COUNT = 1, A_MIN = 2, A_MAX = 3 };

int64_t read_col(const void* data, int32_t type, int64_t i) {
  switch (type) {
    case T_U8: return (int64_t)((const uint8_t*)data)[i];
    case T_I32: return (int64_t)((const int32_t*)data)[i];
    default: return ((const int64_t*)data)[i];
  }
}

int width_bits(int32_t type) { return type == T_U8 ? 8 : type == T_I32 ? 32 : 64; }

template <class T>
T* dup_out(const std::vector<T>& v) {
  T* p = (T*)std::malloc(sizeof(T) * (v.size() ? v.size() : 1));
  if (p && !v.empty()) std::memcpy(p, v.data(), sizeof(T) * v.size());
  return p;
}

}  // namespace

extern "C" {

void orc_free(void* p) { std::free(p); }

// Group key of row i.  One key column: its value (u8 zero-extended, i32 and
// i64 sign-extended).  Several key columns: their bit patterns concatenated,
// first column most significant, each in its own width (8 or 32 bits).
int64_t orc_group_key(int64_t i, int32_t n_keys, const int32_t* key_cols,
                      const void* const* col_data, const int32_t* col_type) {
  if (n_keys == 1) return read_col(col_data[key_cols[0]], col_type[key_cols[0]], i);
  uint64_t k = 0;
  for (int32_t j = 0; j < n_keys; j++) {
    int c = key_cols[j];
    int w = width_bits(col_type[c]);
    uint64_t bits = (uint64_t)read_col(col_data[c], col_type[c], i);
    if (w < 64) bits &= ((uint64_t)1 << w) - 1;
    k = (w < 64 ? (k << w) : 0) | bits;
  }
  return (int64_t)k;
}

// Aggregate input of row i:  base[i] * prod_f (c_f + s_f * fcol_f[i]),
// every product and sum taken mod 2^64.
int64_t orc_agg_value(int64_t i, int32_t base_col, int32_t nf, const int32_t* fcol,
                      const int64_t* c, const int64_t* s, const void* const* col_data,
                      const int32_t* col_type) {
  uint64_t v = (uint64_t)read_col(col_data[base_col], col_type[base_col], i);
  for (int32_t f = 0; f < nf; f++) {
    uint64_t x = (uint64_t)read_col(col_data[fcol[f]], col_type[fcol[f]], i);
    v *= (uint64_t)c[f] + (uint64_t)s[f] * x;
  }
  return (int64_t)v;
}

// Filtered group-by.  A row qualifies when lo_p <= col_p[i] <= hi_p for every
// predicate p.  Each qualifying row joins the group of its key; for each
// aggregate a the group keeps SUM (mod 2^64), COUNT, signed MIN or signed MAX
// of the row's aggregate input (COUNT ignores it).  Only groups with at least
// one qualifying row exist.  Output: groups in ascending signed key order;
// *out_keys = n_groups keys, *out_aggs = n_aggs x n_groups values (aggregate
// major), both malloc'ed (release with orc_free).  Returns n_groups, or -1 on
// allocation failure.
//
// Aggregate a is described by op[a], base[a], nf[a] (0..2) and, for f < nf,
// fcol[2a+f], c[2a+f], s[2a+f].
int64_t orc_groupby(int64_t n_rows, const void* const* col_data, const int32_t* col_type,
                    int32_t n_keys, const int32_t* key_cols, int32_t n_preds,
                    const int32_t* pred_col, const int64_t* pred_lo, const int64_t* pred_hi,
                    int32_t n_aggs, const int32_t* op, const int32_t* base, const int32_t* nf,
                    const int32_t* fcol, const int64_t* c, const int64_t* s,
                    int64_t** out_keys, int64_t** out_aggs) {
  std::unordered_map<int64_t, int64_t> group_of;  // key -> group number
  std::vector<int64_t> keys;                       // group -> key
  std::vector<int64_t> acc;                        // group * n_aggs + a
  for (int64_t i = 0; i < n_rows; i++) {
    bool keep = true;
    for (int32_t p = 0; p < n_preds && keep; p++) {
      int64_t x = read_col(col_data[pred_col[p]], col_type[pred_col[p]], i);
      keep = pred_lo[p] <= x && x <= pred_hi[p];
    }
    if (!keep) continue;
    int64_t k = orc_group_key(i, n_keys, key_cols, col_data, col_type);
    auto it = group_of.find(k);
    int64_t g;
    if (it == group_of.end()) {
      g = (int64_t)keys.size();
      group_of.emplace(k, g);
      keys.push_back(k);
      for (int32_t a = 0; a < n_aggs; a++) {
        int64_t init = 0;
        if (op[a] == A_MIN) init = INT64_MAX;
        if (op[a] == A_MAX) init = INT64_MIN;
        acc.push_back(init);
      }
    } else {
      g = it->second;
    }
    for (int32_t a = 0; a < n_aggs; a++) {
      int64_t& slot = acc[(size_t)(g * n_aggs + a)];
      if (op[a] == A_COUNT) {
        slot += 1;
        continue;
      }
      int64_t v = orc_agg_value(i, base[a], nf[a], fcol + 2 * a, c + 2 * a, s + 2 * a,
                                col_data, col_type);
      switch (op[a]) {
        case A_SUM: slot = (int64_t)((uint64_t)slot + (uint64_t)v); break;
        case A_MIN: slot = std::min(slot, v); break;
        case A_MAX: slot = std::max(slot, v); break;
      }
    }
  }
  int64_t ng = (int64_t)keys.size();
  std::vector<int64_t> order((size_t)ng);
  for (int64_t g = 0; g < ng; g++) order[(size_t)g] = g;
  std::sort(order.begin(), order.end(),
            [&](int64_t x, int64_t y) { return keys[(size_t)x] < keys[(size_t)y]; });
  std::vector<int64_t> ok((size_t)ng), oa((size_t)ng * (size_t)n_aggs);
  for (int64_t r = 0; r < ng; r++) {
    int64_t g = order[(size_t)r];
    ok[(size_t)r] = keys[(size_t)g];
    for (int32_t a = 0; a < n_aggs; a++)
      oa[(size_t)a * (size_t)ng + (size_t)r] = acc[(size_t)(g * n_aggs + a)];
  }
  *out_keys = dup_out(ok);
  *out_aggs = dup_out(oa);
  if (!*out_keys || !*out_aggs) return -1;
  return ng;
}

// Inner equi-join as a bag: every pair (i, j) with probe_key[i] ==
// build_key[j], carrying payload[j] (the gather out = payload[build_idx]).
// Output sorted by (i, j); three malloc'ed columns.  Returns the pair count,
// or -1 on allocation failure.
int64_t orc_join(const int64_t* build_key, const int64_t* payload, int64_t n_build,
                 const int64_t* probe_key, int64_t n_probe, int32_t** out_probe_idx,
                 int32_t** out_build_idx, int64_t** out_payload) {
  std::vector<int32_t> pi, bi;
  std::vector<int64_t> pay;
  if ((double)n_build * (double)n_probe <= (double)(1 << 24)) {
    for (int64_t i = 0; i < n_probe; i++)
      for (int64_t j = 0; j < n_build; j++)
        if (probe_key[i] == build_key[j]) {
          pi.push_back((int32_t)i);
          bi.push_back((int32_t)j);
          pay.push_back(payload[j]);
        }
  } else {
    std::unordered_multimap<int64_t, int32_t> table;
    table.reserve((size_t)n_build);
    for (int64_t j = 0; j < n_build; j++) table.emplace(build_key[j], (int32_t)j);
    std::vector<int32_t> matches;
    for (int64_t i = 0; i < n_probe; i++) {
      auto range = table.equal_range(probe_key[i]);
      matches.clear();
      for (auto it = range.first; it != range.second; ++it) matches.push_back(it->second);
      std::sort(matches.begin(), matches.end());
      for (int32_t j : matches) {
        pi.push_back((int32_t)i);
        bi.push_back(j);
        pay.push_back(payload[j]);
      }
    }
  }
  *out_probe_idx = dup_out(pi);
  *out_build_idx = dup_out(bi);
  *out_payload = dup_out(pay);
  if (!*out_probe_idx || !*out_build_idx || !*out_payload) return -1;
  return (int64_t)pi.size();
}

// Sample summary a planner reads before sizing a group-by (no counterpart in
// the paper; its definition is stated with rel_sketch in include/rel.h):
// the sample is every row when n_rows <= 4096, else rows
// floor(w * (n_rows - 64) / 63) + o for w, o in [0, 64); filtered rows are
// dropped.  Writes, in order: sample_rows, kept, ndv, singletons, runs into
// ints[0..5); key_min, key_max into mm[0..2); top keys / counts (count
// descending, key ascending, up to 32); the 256 HyperLogLog registers.
void orc_sketch(int64_t n_rows, const void* const* col_data, const int32_t* col_type,
                int32_t n_keys, const int32_t* key_cols, int32_t n_preds,
                const int32_t* pred_col, const int64_t* pred_lo, const int64_t* pred_hi,
                int32_t* ints, int64_t* mm, int64_t* top_key, int32_t* top_count,
                uint8_t* hll) {
  const int64_t S = n_rows < 4096 ? n_rows : 4096;
  std::vector<int64_t> kept_keys;
  std::vector<int> block;  // which block of 64 sample positions a kept key came from
  for (int64_t j = 0; j < S; j++) {
    const int64_t row = n_rows <= 4096 ? j : (j / 64) * (n_rows - 64) / 63 + (j % 64);
    bool keep = true;
    for (int32_t p = 0; p < n_preds && keep; p++) {
      int64_t x = read_col(col_data[pred_col[p]], col_type[pred_col[p]], row);
      keep = pred_lo[p] <= x && x <= pred_hi[p];
    }
    if (!keep) continue;
    kept_keys.push_back(orc_group_key(row, n_keys, key_cols, col_data, col_type));
    block.push_back((int)(j / 64));
  }
  std::memset(hll, 0, 256);
  for (int64_t k : kept_keys) {
    // splitmix64 output function of the key (Steele, Lea & Flood 2014)
    uint64_t z = (uint64_t)k + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const int reg = (int)(z >> 56);
    uint64_t rest = z << 8;  // the other 56 bits, at the top of the word
    int rank = 1;
    if (rest == 0) {
      rank = 57;
    } else {
      while (!(rest >> 63)) {
        rest <<= 1;
        rank++;
      }
    }
    if (rank > hll[reg]) hll[reg] = (uint8_t)rank;
  }
  std::unordered_map<int64_t, int32_t> count;
  for (int64_t k : kept_keys) count[k] += 1;
  int runs = 0;
  for (size_t i = 0; i < kept_keys.size(); i++)
    if (i == 0 || block[i] != block[i - 1] || kept_keys[i] != kept_keys[i - 1]) runs++;
  int singles = 0;
  std::vector<std::pair<int32_t, int64_t>> byfreq;
  for (auto& kv : count) {
    if (kv.second == 1) singles++;
    byfreq.push_back({kv.second, kv.first});
  }
  std::sort(byfreq.begin(), byfreq.end(), [](const auto& a, const auto& b) {
    return a.first != b.first ? a.first > b.first : a.second < b.second;
  });
  for (int i = 0; i < 32; i++) {
    top_key[i] = i < (int)byfreq.size() ? byfreq[(size_t)i].second : 0;
    top_count[i] = i < (int)byfreq.size() ? byfreq[(size_t)i].first : 0;
  }
  ints[0] = (int32_t)S;
  ints[1] = (int32_t)kept_keys.size();
  ints[2] = (int32_t)count.size();
  ints[3] = singles;
  ints[4] = runs;
  mm[0] = kept_keys.empty() ? 0 : *std::min_element(kept_keys.begin(), kept_keys.end());
  mm[1] = kept_keys.empty() ? 0 : *std::max_element(kept_keys.begin(), kept_keys.end());
}

// Number of pairs the join above emits (the paper's "count" step).
int64_t orc_join_count(const int64_t* build_key, int64_t n_build, const int64_t* probe_key,
                       int64_t n_probe) {
  std::unordered_map<int64_t, int64_t> mult;
  mult.reserve((size_t)n_build);
  for (int64_t j = 0; j < n_build; j++) mult[build_key[j]] += 1;
  int64_t total = 0;
  for (int64_t i = 0; i < n_probe; i++) {
    auto it = mult.find(probe_key[i]);
    if (it != mult.end()) total += it->second;
  }
  return total;
}

}  // extern "C"
