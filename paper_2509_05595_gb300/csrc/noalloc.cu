// pamo_check_self_intersections_noalloc: the self-intersection check without
// any device allocation.
//
// Some callers cannot call cudaMalloc: code that must not grow its device
// footprint or block on the allocator while it runs (for example a service
// whose device memory is owned and budgeted by another component, or a
// latency-bound loop that has reserved everything up front).  For them this
// entry point runs the same LBVH + exact narrow phase as
// pamo_check_self_intersections, with every scratch buffer carved out of one
// file-scope device array of fixed size, which each GPU that loads the library
// holds until the process exits.  The caller still provides the mesh and the
// output pair buffer.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "common.cuh"

namespace pamo {
namespace {

constexpr int64_t kMaxFaces = 32768;
constexpr int64_t kMaxVertices = 32768;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte layout of the scratch for the maximum sizes (256-byte aligned pieces).
struct Layout {
  size_t pos, F, dc, bad, bbox, nodes, parent, flags, keys, vals, keys2, vals2, hist, aux, len,
      sums, total;
  size_t nodes_b, parent_b, flags_b, kv_b, hist_b, aux_b, sums_b;
};

constexpr size_t kTiles = (kMaxFaces + kSortTile - 1) / kSortTile;  // radix-sort tiles

constexpr Layout make_layout() {
  Layout L{};
  L.nodes_b = sizeof(float) * 24 * (size_t)kMaxFaces;  // nodes, then leaf boxes
  L.parent_b = sizeof(int32_t) * (size_t)(2 * kMaxFaces + 1);
  L.flags_b = sizeof(int32_t) * (size_t)(kMaxFaces + 2);
  L.kv_b = sizeof(uint32_t) * (size_t)kMaxFaces;
  L.hist_b = sizeof(int32_t) * (size_t)(2 * 256 * kTiles + 2);
  L.aux_b = (size_t)kMaxFaces + 16;
  // tile sums of the prefix scans, total after them
  L.sums_b = sizeof(int32_t) * (size_t)((kMaxFaces + kScanTile - 1) / kScanTile + 1);
  size_t o = 0;
  L.pos = o; o += align256(sizeof(float) * 4 * (size_t)kMaxVertices);
  L.F = o; o += align256(sizeof(int) * 4 * (size_t)kMaxFaces);
  L.dc = o; o += align256(sizeof(RoundCounters));
  L.bad = o; o += align256(sizeof(int));
  L.bbox = o; o += align256(6 * sizeof(unsigned));
  L.nodes = o; o += align256(L.nodes_b);
  L.parent = o; o += align256(L.parent_b);
  L.flags = o; o += align256(L.flags_b);
  L.keys = o; o += align256(L.kv_b);
  L.vals = o; o += align256(L.kv_b);
  L.keys2 = o; o += align256(L.kv_b);
  L.vals2 = o; o += align256(L.kv_b);
  L.hist = o; o += align256(L.hist_b);
  L.aux = o; o += align256(L.aux_b);
  L.len = o; o += align256(16);
  L.sums = o; o += align256(L.sums_b);
  L.total = o;
  return L;
}

constexpr Layout kL = make_layout();

// The scratch (about 4.9 MiB).  In host code this name is only a host-side
// stand-in: kernels get the device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kL.total];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device, looked up once per
// device (the first call on each device does this set-up).
pamo_status scratch_address(unsigned char** out) {
  int dev = -1;
  PAMO_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range for the scratch table");
    return PAMO_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scratch)");
    g_addr[dev] = p;
  }
  *out = (unsigned char*)g_addr[dev];
  return PAMO_OK;
}

}  // namespace
}  // namespace pamo

using namespace pamo;

extern "C" pamo_status pamo_check_self_intersections_noalloc(const float* d_V, int64_t nV,
                                                             const int32_t* d_F, int64_t nF,
                                                             void* stream, int64_t* n_pairs,
                                                             int32_t* d_pairs, int64_t cap) {
  if (!d_V || !d_F || !n_pairs || nV <= 0 || nF <= 0 || cap < 0 || (cap > 0 && !d_pairs)) {
    set_error("device mesh, n_pairs and (for cap > 0) d_pairs required");
    return PAMO_EINVAL;
  }
  if (nF > kMaxFaces || nV > kMaxVertices) {
    set_error("pamo_check_self_intersections_noalloc: mesh too large for the fixed scratch "
              "(at most 32768 faces and 32768 vertices); use pamo_check_self_intersections");
    return PAMO_EINVAL;
  }
  {  // the fixed layout must cover what the BVH passes index for this size
    size_t nb, pb, fb, kvb, hb, ab;
    int64_t hw;
    bvh_bytes((int)nF, &nb, &pb, &fb, &kvb, &hb, &ab, &hw);
    if (nb > kL.nodes_b || pb > kL.parent_b || fb > kL.flags_b || kvb > kL.kv_b ||
        hb > kL.hist_b || ab > kL.aux_b ||
        (size_t)scan_sums_count(hw > nF ? hw : nF) * sizeof(int32_t) > kL.sums_b) {
      set_error("internal: scratch layout smaller than the BVH needs");
      return PAMO_EINTERNAL;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  PAMO_TRY(scratch_address(&base));
  float4* pos = (float4*)(base + kL.pos);
  int4* F = (int4*)(base + kL.F);
  RoundCounters* dc = (RoundCounters*)(base + kL.dc);
  Bvh b;
  b.nodes = Buf{base + kL.nodes, kL.nodes_b};
  b.parent = Buf{base + kL.parent, kL.parent_b};
  b.flags = Buf{base + kL.flags, kL.flags_b};
  b.keys = Buf{base + kL.keys, kL.kv_b};
  b.vals = Buf{base + kL.vals, kL.kv_b};
  b.keys2 = Buf{base + kL.keys2, kL.kv_b};
  b.vals2 = Buf{base + kL.vals2, kL.kv_b};
  b.hist = Buf{base + kL.hist, kL.hist_b};
  b.face_aux = Buf{base + kL.aux, kL.aux_b};
  b.sort_len = Buf{base + kL.len, 16};
  b.sums = Buf{base + kL.sums, kL.sums_b};
  b.n_max = (int)nF;
  // the array keeps the previous call's contents: the counters must start at 0
  PAMO_CUDA(cudaMemsetAsync(dc, 0, sizeof(RoundCounters), st));
  // every face index is checked against [0, nV) before anything reads the mesh
  PAMO_TRY(load_mesh_checked(d_V, nV, d_F, nF, pos, F, (int*)(base + kL.bad), st));
  float lo[3], hi[3];
  PAMO_TRY(mesh_bbox_into(pos, nV, (unsigned*)(base + kL.bbox), lo, hi, st));
  PAMO_TRY(bvh_build(b, pos, F, nullptr, nullptr, (int)nF, lo, hi, false, default_grid(), st));
  PAMO_TRY(bvh_check(b, pos, F, nullptr, nullptr, 1, nullptr, nullptr, 0, nullptr, dc, d_pairs,
                     cap, (int)nF, st));
  RoundCounters h;
  std::memset(&h, 0, sizeof(h));
  PAMO_CUDA(cudaMemcpyAsync(&h, dc, sizeof(h), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  if (h.overflow) {
    set_error("BVH traversal stack overflow");
    return PAMO_EINTERNAL;
  }
  *n_pairs = h.n_pairs;
  return PAMO_OK;
}
