// rel_groupby_agg_static: the group-by for callers that cannot allocate
// device memory.
//
// Some callers have no way to obtain the workspace rel_groupby_agg asks for:
// an engine that hands all device memory to its own pool and forbids any
// other allocation, a plugin running under a host process that caps device
// memory, or a latency-critical path where cudaMalloc / cudaFree (which can
// synchronise the whole device) are not acceptable.  This entry point lets
// them aggregate anyway: the hash table lives in a fixed array compiled into
// the library, so the call itself allocates nothing.  The caller still
// provides the input columns and the output arrays.
//
// The array is a file-scope __device__ variable: every GPU on which the
// library is loaded holds its STATIC_WS_BYTES (about 4.5 MiB) until the
// process exits.  Host code must not hand the array's name to a kernel -- on
// the host that name is only a stand-in, not a device address -- so every
// call looks up the device address with cudaGetSymbolAddress, with the
// caller's device current.  The lookup is cheap next to the kernels, and a
// fresh one stays valid after a cudaDeviceReset reloaded the module.
#include "rel_internal.cuh"

namespace {

constexpr int64_t STATIC_MAX_GROUPS = REL_STATIC_MAX_GROUPS;
constexpr int64_t STATIC_SLOTS = 2 * STATIC_MAX_GROUPS;  // load factor <= 1/2
constexpr size_t STATIC_WS_BYTES =
    rel::HEADER_BYTES + (size_t)STATIC_SLOTS * 8u * (1u + REL_MAX_AGGS);

// Workspace shared by every call on a device: header, keys, aggregate words.
static __device__ __align__(256) unsigned char g_static_ws[STATIC_WS_BYTES];

// Device address of g_static_ws on the current device.
rel_status static_ws_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
  *out = p;
  return REL_OK;
}

}  // namespace

extern "C" rel_status rel_groupby_agg_static(const rel_groupby_desc* desc, int64_t max_groups,
                                             int64_t* out_keys, int64_t* const* out_aggs,
                                             int64_t out_capacity, int64_t* n_groups_host,
                                             void* stream) {
  if (max_groups < 1 || max_groups > STATIC_MAX_GROUPS) {
    relhost::set_error(
        "static group-by: max_groups = %lld is outside 1..%lld, the most the built-in "
        "%zu-byte scratch table holds; use rel_groupby_agg with a caller workspace",
        (long long)max_groups, (long long)STATIC_MAX_GROUPS, STATIC_WS_BYTES);
    return REL_E_UNSUPPORTED;
  }
  // Overflow of the fixed table is only detected by reading the status back,
  // which needs the host count: without it a caller could get a truncated
  // result reported as success.
  if (!n_groups_host) {
    relhost::set_error("static group-by: n_groups_host must not be NULL (it carries the "
                       "group count and the overflow check)");
    return REL_E_INVALID;
  }
  // Host-only sizing: a positive hint makes rel_plan_size touch no device.
  rel_plan plan;
  rel_status r = rel_plan_size(REL_OP_GROUPBY, desc, 0u, max_groups, nullptr, 0, &plan, stream);
  if (r != REL_OK) return r;
  if (plan.variant == REL_VAR_PARTITIONED) {
    // the partitioned variant keeps a record per input row: too much for a
    // fixed array, so stay with the layered single table
    plan.variant = REL_VAR_GLOBAL;
    plan.part_bits = 0;
    plan.tiny_slots = 8;
    plan.smem_slots = 2048;
    plan.workspace_bytes = rel_groupby_ws_bytes(plan.slots, desc->n_aggs);
  }
  if (plan.workspace_bytes > STATIC_WS_BYTES) {
    relhost::set_error("static group-by: plan needs %llu bytes, scratch holds %zu",
                       (unsigned long long)plan.workspace_bytes, STATIC_WS_BYTES);
    return REL_E_UNSUPPORTED;
  }
  void* ws = nullptr;
  if ((r = static_ws_address(&ws)) != REL_OK) return r;
  // rel_groupby_agg clears the part of the workspace it uses before its kernels run.
  return rel_groupby_agg(desc, &plan, ws, STATIC_WS_BYTES, out_keys, out_aggs, out_capacity,
                         n_groups_host, stream);
}
