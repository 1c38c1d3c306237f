// Intersection check of Section 5.2 / Algorithm 3: a linear BVH over the
// faces (Karras 2012: Morton codes of the face-box centres, a radix sort, the
// binary radix tree built in parallel, boxes refitted bottom-up), queried
// with the faces that changed this round.  Candidate pairs (closed boxes
// overlap) are written to three buckets by their number of shared vertices
// (k_traverse) and tested by the exact narrow phase (exact.cuh) one thread per
// pair (k_pairs), so a warp follows one branch of Algorithm 3; when a bucket
// overflows, the fused traversal + narrow phase (k_query) reruns the check.
//
// Face boxes are the min/max of float32 corner coordinates, which is exact,
// and overlap is tested on closed intervals, so the broad phase never drops a
// touching pair.
#include <utility>

#include "common.cuh"
#include "exact.cuh"

namespace pamo {

namespace {

constexpr int kSortItems = kSortTile / kBlock;  // 4096 keys per block
// Traversal stack.  Along any root-to-leaf path of the radix tree the common
// prefix length of the node's key range grows strictly, and the prefixes are
// drawn from at most 31 Morton bits (30 plus the dead-face bit) and, among
// equal Morton keys, at most 31 bits of the leaf index (n < 2^30 faces): a
// path has at most 62 internal nodes.  A query pushes at most one node per
// level it descends, so 64 entries always suffice (in a batch each query
// starts at its own mesh's subtree root, below the mesh-id levels).
constexpr int kStack = 64;

__device__ __forceinline__ unsigned spread10(unsigned x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__device__ __forceinline__ unsigned quant(float c, float lo, float inv) {
  float t = (c - lo) * inv;
  t = fminf(fmaxf(t, 0.0f), 1.0f);
  return (unsigned)(t * 1023.0f);
}

__device__ __forceinline__ uint8_t pack_info(exact::FaceInfo fi) {
  return (uint8_t)(fi.axis * 3 + (fi.o + 1));
}
__device__ __forceinline__ exact::FaceInfo unpack_info(uint8_t b) {
  exact::FaceInfo fi;
  fi.axis = b / 3;
  fi.o = (int)(b % 3) - 1;
  return fi;
}

#define GRID_STRIDE(i, n) \
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

// Morton keys of the face-box centres and the identity leaf order (the boxes
// and the faces' predicate info are written by the refit, after the sort).
// Many meshes in one tree (a batch): the key of a leaf is (mesh id, Morton code
// in that mesh's own frame), the mesh id in the high word hkeys, so the radix
// tree separates the meshes before any spatial split and every mesh owns a
// subtree (its root in mroot); mframe holds each mesh's frame (lo.xyz,
// 1/extent.xyz).  With vmesh == nullptr there is one mesh and no high word.
__global__ void k_leaf_keys(const float4* __restrict__ pos, const int4* __restrict__ F,
                            const uint8_t* __restrict__ fdead, const int* n_dev, int n_host,
                            float lx, float ly, float lz, float ix, float iy, float iz,
                            const int32_t* __restrict__ vmesh, const float* __restrict__ mframe,
                            unsigned* __restrict__ keys, unsigned* __restrict__ hkeys,
                            int32_t* __restrict__ vals) {
  const int n = dev_n(n_dev, n_host);
  GRID_STRIDE(f, n) {
  vals[f] = f;
  const int4 t = F[f];
  if (vmesh) {
    const int m = vmesh[t.x];
    hkeys[f] = (unsigned)m;
    lx = mframe[6 * m]; ly = mframe[6 * m + 1]; lz = mframe[6 * m + 2];
    ix = mframe[6 * m + 3]; iy = mframe[6 * m + 4]; iz = mframe[6 * m + 5];
  }
  if (fdead && fdead[f]) {
    keys[f] = 1u << 30;
    continue;
  }
  const float4 a = pos[t.x], b = pos[t.y], c = pos[t.z];
  const float cx = 0.5f * (fminf(fminf(a.x, b.x), c.x) + fmaxf(fmaxf(a.x, b.x), c.x));
  const float cy = 0.5f * (fminf(fminf(a.y, b.y), c.y) + fmaxf(fmaxf(a.y, b.y), c.y));
  const float cz = 0.5f * (fminf(fminf(a.z, b.z), c.z) + fmaxf(fmaxf(a.z, b.z), c.z));
  keys[f] = (spread10(quant(cx, lx, ix)) << 2) | (spread10(quant(cy, ly, iy)) << 1) |
            spread10(quant(cz, lz, iz));
  }
}

// ---- LSD radix sort of (key, value), 8 bits per pass, stable -------------
__device__ __forceinline__ int sort_tiles(int n) { return n > 0 ? (n + kSortTile - 1) / kSortTile : 1; }

// scan length of the digit histogram (256 digits x tiles), for the scan
__global__ void k_sort_len(const int* n_dev, int n_host, int* __restrict__ len) {
  *len = 256 * sort_tiles(dev_n(n_dev, n_host));
}

// keys: the array the digit of this pass is taken from (Morton or mesh word)
__global__ void k_digit_hist(const unsigned* __restrict__ keys, const int* n_dev, int n_host,
                             int shift, int32_t* __restrict__ hist) {
  __shared__ int h[256];
  const int n = dev_n(n_dev, n_host);
  const int tiles = sort_tiles(n);
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = tile * kSortTile;
#pragma unroll 4
    for (int i = 0; i < kSortItems; i++) {
      const int j = base + i * kBlock + threadIdx.x;
      if (j < n) atomicAdd(&h[(keys[j] >> shift) & 0xffu], 1);
    }
    __syncthreads();
    hist[threadIdx.x * tiles + tile] = h[threadIdx.x];
    __syncthreads();
  }
}

// moves (key, value[, high word]); the digit comes from the high word when
// from_hi is set
__global__ void __launch_bounds__(kBlock) k_digit_scatter(
    const unsigned* __restrict__ keys, const int32_t* __restrict__ vals,
    const unsigned* __restrict__ hk, int from_hi, const int* n_dev,
    int n_host, int shift, const int32_t* __restrict__ offs, unsigned* __restrict__ okeys,
    int32_t* __restrict__ ovals, unsigned* __restrict__ ohk) {
  __shared__ int wcount[kBlock / 32][256];
  __shared__ int goff[256];
  const int n = dev_n(n_dev, n_host);
  const int tiles = sort_tiles(n);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
  for (int i = threadIdx.x; i < (kBlock / 32) * 256; i += kBlock) (&wcount[0][0])[i] = 0;
  goff[threadIdx.x] = offs[threadIdx.x * tiles + tile];
  __syncthreads();
  const int base = tile * kSortTile + wid * (kSortItems * 32);
  unsigned k[kSortItems], h[kSortItems];
  int v[kSortItems], r[kSortItems];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const int j = base + i * 32 + lane;
    const bool ok = j < n;
    k[i] = ok ? keys[j] : 0u;
    v[i] = ok ? vals[j] : 0;
    h[i] = (ok && hk) ? hk[j] : 0u;
    const unsigned src = from_hi ? h[i] : k[i];
    const unsigned d = ok ? ((src >> shift) & 0xffu) : (0x100u | lane);
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    int before = 0;
    if (ok) before = wcount[wid][d];
    r[i] = before + __popc(peers & lt);
    __syncwarp();
    if (ok && (peers & lt) == 0) wcount[wid][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // exclusive prefix over warps for each digit
    int run = 0;
    for (int w = 0; w < kBlock / 32; w++) {
      int t = wcount[w][threadIdx.x];
      wcount[w][threadIdx.x] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSortItems; i++) {
    const int j = base + i * 32 + lane;
    if (j < n) {
      const unsigned d = ((from_hi ? h[i] : k[i]) >> shift) & 0xffu;
      const int p = goff[d] + wcount[wid][d] + r[i];
      okeys[p] = k[i];
      ovals[p] = v[i];
      if (hk) ohk[p] = h[i];
    }
  }
  __syncthreads();
  }
}

// ---- Karras binary radix tree ---------------------------------------------
// common prefix length of the keys (high word, Morton word, then index for
// equal keys), -1 outside [0, n)
__device__ __forceinline__ int delta(const unsigned* __restrict__ k,
                                     const unsigned* __restrict__ hk, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  if (hk) {
    const unsigned ha = hk[i], hb = hk[j];
    if (ha != hb) return __clz(ha ^ hb);
  }
  const unsigned a = k[i], b = k[j];
  if (a == b) return 64 + __clz(i ^ j);
  return 32 + __clz(a ^ b);
}

// Node layout (64 bytes, internal nodes only): the boxes of both children and
// the child links, so that one 64-byte load serves a whole traversal level.
//   floats 0-5:  left child box  (lo.xyz, hi.xyz)
//   floats 6-11: right child box (lo.xyz, hi.xyz)
//   ints 12, 13: left, right child (internal index >= 0, or ~face for a leaf)
//   ints 14, 15: the node's leaf range [first, last] (read by the refit)
// parent[x] = (parent node << 1) | side for internal x in [0, n-1) and leaf
// positions x = n-1+j; the root has -1.
// With high words (a batch), the node whose range is exactly one mesh's
// leaves is that mesh's subtree root (mroot).
__global__ void k_karras(const unsigned* __restrict__ k, const unsigned* __restrict__ hk,
                         const int32_t* __restrict__ vals, const int* n_dev, int n_host,
                         float* __restrict__ nodes, int32_t* __restrict__ parent,
                         int32_t* __restrict__ mroot) {
  const int n = dev_n(n_dev, n_host);
  GRID_STRIDE(i, n - 1) {
  const int d = (delta(k, hk, n, i, i + 1) - delta(k, hk, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = delta(k, hk, n, i, i - d);
  int lmax = 2;
  while (delta(k, hk, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(k, hk, n, i, i + (l + t) * d) > dmin) l += t;
  const int j = i + l * d;
  const int dnode = delta(k, hk, n, i, j);
  int s = 0;
  for (int div = 2;; div <<= 1) {
    const int t = (l + div - 1) / div;
    if (delta(k, hk, n, i, i + (s + t) * d) > dnode) s += t;
    if (t <= 1) break;
  }
  if (hk) {
    const int first = min(i, j), last = max(i, j);
    const unsigned m = hk[first];
    if (hk[last] == m && (first == 0 || hk[first - 1] != m) && (last == n - 1 || hk[last + 1] != m))
      mroot[m] = i;
  }
  const int g = i + s * d + (d < 0 ? -1 : 0);
  const bool lleaf = min(i, j) == g, rleaf = max(i, j) == g + 1;
  const int left = lleaf ? ~vals[g] : g;
  const int right = rleaf ? ~vals[g + 1] : g + 1;
  int* links = reinterpret_cast<int*>(nodes + 16 * (size_t)i + 12);
  links[0] = left;
  links[1] = right;
  links[2] = min(i, j);
  links[3] = max(i, j);
  parent[lleaf ? n - 1 + g : g] = (i << 1) | 0;
  parent[rleaf ? n - 1 + g + 1 : g + 1] = (i << 1) | 1;
  if (i == 0) parent[0] = -1;
  }
}

__global__ void k_order_write(const int32_t* __restrict__ vals, const unsigned* __restrict__ keys,
                              const unsigned* __restrict__ hk, const int* n_dev,
                              const uint8_t* __restrict__ fdead, const int32_t* __restrict__ pos,
                              const int32_t* __restrict__ dead_before, int32_t* __restrict__ out,
                              unsigned* __restrict__ okeys, unsigned* __restrict__ ohk) {
  const int n = *n_dev;
  GRID_STRIDE(i, n) {
    const int f = vals[i];
    if (fdead[f]) continue;
    out[pos[i]] = f - dead_before[f];
    okeys[pos[i]] = keys[i];
    if (hk) ohk[pos[i]] = hk[i];
  }
}

__global__ void k_copy_order(const int32_t* __restrict__ vals2, const unsigned* __restrict__ keys2,
                             const unsigned* __restrict__ hk2, const int* n_dev, int n_host,
                             int32_t* __restrict__ vals, unsigned* __restrict__ keys,
                             unsigned* __restrict__ hk) {
  const int n = dev_n(n_dev, n_host);
  GRID_STRIDE(i, n) {
    vals[i] = vals2[i];
    keys[i] = keys2[i];
    if (hk) hk[i] = hk2[i];
  }
}

__device__ __forceinline__ void store_box(float* __restrict__ nodes, int p, int side,
                                          const float3& lo, const float3& hi) {
  float2* dst = reinterpret_cast<float2*>(nodes + 16 * (size_t)p + 6 * side);
  dst[0] = make_float2(lo.x, lo.y);
  dst[1] = make_float2(lo.z, hi.x);
  dst[2] = make_float2(hi.y, hi.z);
}

// atomic add with acquire-release semantics at device scope
__device__ __forceinline__ int add_acq_rel(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;"
               : "=r"(old)
               : "l"(p), "r"(v)
               : "memory");
  return old;
}

// Leaf boxes in leaf order (lo.xyz, hi.xyz as two float4; a dead face's box
// is empty), and each face's predicate info (dominant normal axis and
// orientation, read by the exact pair test) from the corners loaded for it.
__global__ void k_leaf_boxes(const float4* __restrict__ pos, const int4* __restrict__ F,
                             const uint8_t* __restrict__ fdead, const int32_t* __restrict__ vals,
                             const int* n_dev, int n_host, float4* __restrict__ lbox,
                             uint8_t* __restrict__ info) {
  const int n = dev_n(n_dev, n_host);
  GRID_STRIDE(j, n) {
    const int f = vals[j];
    float3 lo, hi;
    if (fdead && fdead[f]) {
      lo = make_float3(INFINITY, INFINITY, INFINITY);
      hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
      info[f] = pack_info(exact::FaceInfo{0, 0});
    } else {
      const int4 t = F[f];
      const float4 a = pos[t.x], b = pos[t.y], c = pos[t.z];
      lo = make_float3(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y),
                       fminf(fminf(a.z, b.z), c.z));
      hi = make_float3(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y),
                       fmaxf(fmaxf(a.z, b.z), c.z));
      info[f] = pack_info(exact::face_info(make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z),
                                           make_float3(c.x, c.y, c.z)));
    }
    lbox[2 * (size_t)j] = make_float4(lo.x, lo.y, lo.z, 0.f);
    lbox[2 * (size_t)j + 1] = make_float4(hi.x, hi.y, hi.z, 0.f);
  }
}

// union of the leaf boxes [a, b]
__device__ __forceinline__ void range_box(const float4* __restrict__ lbox, int a, int b,
                                          float3& lo, float3& hi) {
  float4 l = lbox[2 * (size_t)a], h = lbox[2 * (size_t)a + 1];
  for (int j = a + 1; j <= b; j++) {
    const float4 l2 = lbox[2 * (size_t)j], h2 = lbox[2 * (size_t)j + 1];
    l.x = fminf(l.x, l2.x); l.y = fminf(l.y, l2.y); l.z = fminf(l.z, l2.z);
    h.x = fmaxf(h.x, h2.x); h.y = fmaxf(h.y, h2.y); h.z = fmaxf(h.z, h2.z);
  }
  lo = make_float3(l.x, l.y, l.z);
  hi = make_float3(h.x, h.y, h.z);
}

// Internal-node boxes, one thread per node (6 blocks of 256 per SM).  A child
// covering at most kRefitLeaves leaves (or one leaf) gets its box straight from
// the leaf boxes, with no ordering against other threads; most nodes lie in
// the bottom levels, so most boxes come this way.  Only nodes covering more leaves than that wait
// for their children: each such node counts two arrivals, one per child (its
// own thread arrives for a child it filled itself, a child's climb for a
// larger child), with a release-acquire counter, and the second arrival
// computes the node's box, stores it in the parent and climbs on.  Box values
// are min/max of the same leaf boxes as any bottom-up order, so they are
// identical to a leaf-by-leaf climb.
constexpr int kRefitLeaves = 16;
__global__ void __launch_bounds__(kBlock, 6)
    k_refit_nodes(const float4* __restrict__ lbox, const int* n_dev, int n_host,
                  float* __restrict__ nodes, const int32_t* __restrict__ parent,
                  int32_t* __restrict__ flags, int* __restrict__ overflow) {
  const int n = dev_n(n_dev, n_host);
  if (n < 2) return;
  GRID_STRIDE(i, n - 1) {
    const int4 t = *reinterpret_cast<const int4*>(nodes + 16 * (size_t)i + 12);
    const int first = t.z, last = t.w;
    const int g = t.x >= 0 ? t.x : first;  // the left child covers [first, g]
    const bool lsmall = g - first + 1 <= kRefitLeaves, rsmall = last - g <= kRefitLeaves;
    float3 lo, hi;
    if (lsmall) {
      range_box(lbox, first, g, lo, hi);
      store_box(nodes, i, 0, lo, hi);
    }
    if (rsmall) {
      range_box(lbox, g + 1, last, lo, hi);
      store_box(nodes, i, 1, lo, hi);
    }
    // a node this small is read by its parent from the leaves directly
    if (last - first + 1 <= kRefitLeaves) continue;
    const int own = (int)lsmall + (int)rsmall;
    if (own == 0) continue;  // both children larger: their climbs complete this node
    // one side filled here: arrive for it (release); the second arrival goes on
    if (own == 1 && add_acq_rel(&flags[i], 1) == 0) continue;
    int p = i;
    // a radix tree over n leaves is at most n - 1 levels deep; the cap only
    // guards against a malformed tree
    for (int steps = 0;; steps++) {
      if (steps >= n) {
        atomicOr(overflow, 2);
        break;
      }
      const int ps = parent[p];
      if (ps < 0) break;  // root: its box is never needed
      const float4* q = reinterpret_cast<const float4*>(nodes + 16 * (size_t)p);
      const float4 a = __ldcg(q), b = __ldcg(q + 1), c = __ldcg(q + 2);
      lo = make_float3(fminf(a.x, b.z), fminf(a.y, b.w), fminf(a.z, c.x));
      hi = make_float3(fmaxf(a.w, c.y), fmaxf(b.x, c.z), fmaxf(b.y, c.w));
      store_box(nodes, ps >> 1, ps & 1, lo, hi);
      p = ps >> 1;
      // arrival count with release (our box store is visible before the count)
      // and acquire (the sibling's box is visible to the second arrival)
      if (add_acq_rel(&flags[p], 1) == 0) break;  // sibling not ready: it finishes
    }
  }
}

// start of a split check: zero the pair / undo / candidate counters and fold
// a refit overflow into the round's overflow word; a re-check also moves its
// query window to the faces the last undo restored
__global__ void k_check_begin(const int32_t* __restrict__ refit_overflow,
                              RoundCounters* __restrict__ dc, int advance) {
  if (advance) {
    dc->rest_lo = dc->rest_mid;
    dc->rest_mid = dc->rest_end;
  }
  dc->n_pairs = 0;
  dc->n_undo = 0;
  dc->ncand[0] = dc->ncand[1] = dc->ncand[2] = 0;
  dc->cand_overflow = 0;
  if (*refit_overflow) atomicOr(&dc->overflow, *refit_overflow);
}

__global__ void k_fold_overflow(const int32_t* __restrict__ src, int* __restrict__ dst) {
  if (*src) atomicOr(dst, *src);
}

__device__ __forceinline__ bool overlap(const float3& alo, const float3& ahi, float blx, float bly,
                                        float blz, float bhx, float bhy, float bhz) {
  return !(alo.x > bhx || blx > ahi.x || alo.y > bhy || bly > ahi.y || alo.z > bhz || blz > ahi.z);
}

__device__ __forceinline__ float3 sub3f(const float4& a, const float4& b) {
  return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 cross3f(const float3& a, const float3& b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// one 64-byte node: which children overlap the query box, and their links
struct NodeHits {
  bool l, r;
  int L, R;
};

__device__ __forceinline__ NodeHits visit(const float* __restrict__ nodes, int node,
                                          const float3& lo, const float3& hi) {
  const float4* q = reinterpret_cast<const float4*>(nodes + 16 * (size_t)node);
  const float4 a = q[0], b = q[1], c = q[2], d = q[3];
  NodeHits h;
  h.l = overlap(lo, hi, a.x, a.y, a.z, a.w, b.x, b.y);
  h.r = overlap(lo, hi, b.z, b.w, c.x, c.y, c.z, c.w);
  h.L = __float_as_int(d.x);
  h.R = __float_as_int(d.y);
  return h;
}

// One thread per query face.  Query faces: every live face when query_all,
// else the faces with ftag[f] >= 0 (changed this round).  A pair of two query
// faces is evaluated once, from its lower face id.  Intersecting pairs mark
// the collapses that tagged either face.
__global__ void __launch_bounds__(kBlock) k_query(
    const float* __restrict__ nodes, const int* n_dev, int n_host, const float4* __restrict__ pos,
    const int4* __restrict__ F, const uint8_t* __restrict__ fdead,
    const uint8_t* __restrict__ info, const int32_t* __restrict__ ftag, int query_all,
    const int32_t* __restrict__ qlist, const int* __restrict__ qcount,
    uint8_t* __restrict__ undo, RoundCounters* __restrict__ dc, int32_t* __restrict__ pairs_out,
    int64_t cap, const int32_t* __restrict__ vmesh, const int32_t* __restrict__ mroot) {
  const int n = dev_n(n_dev, n_host);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int f;
  if (query_all) {
    if (i >= n) return;
    f = i;
  } else {
    if (i >= *qcount) return;
    f = qlist[i];
  }
  if (fdead && fdead[f]) return;
  const int tf = ftag ? ftag[f] : -1;
  if (!query_all && tf < 0) return;
  const int4 tv = F[f];
  const int ti[3] = {tv.x, tv.y, tv.z};
  float3 T[3];
  {
    const float4 a = pos[tv.x], b = pos[tv.y], c = pos[tv.z];
    T[0] = make_float3(a.x, a.y, a.z);
    T[1] = make_float3(b.x, b.y, b.z);
    T[2] = make_float3(c.x, c.y, c.z);
  }
  const float3 lo = make_float3(fminf(fminf(T[0].x, T[1].x), T[2].x),
                                fminf(fminf(T[0].y, T[1].y), T[2].y),
                                fminf(fminf(T[0].z, T[1].z), T[2].z));
  const float3 hi = make_float3(fmaxf(fmaxf(T[0].x, T[1].x), T[2].x),
                                fmaxf(fmaxf(T[0].y, T[1].y), T[2].y),
                                fmaxf(fmaxf(T[0].z, T[1].z), T[2].z));
  const exact::FaceInfo fiT = unpack_info(info[f]);
  int stack[kStack];
  int sp = 0;
  if (n == 1) return;
  int node = mroot ? mroot[vmesh[tv.x]] : 0;  // the query's own mesh
  // a tree has 2n - 1 nodes; the visit cap only guards against a malformed one
  for (int visits = 0;; visits++) {
    if (visits >= 2 * n) {
      atomicOr(&dc->overflow, 4);
      return;
    }
    const NodeHits h = visit(nodes, node, lo, hi);
    int next = -1;
#pragma unroll
    for (int c = 0; c < 2; c++) {
      if (!(c ? h.r : h.l)) continue;
      const int cn = c ? h.R : h.L;
      if (cn < 0) {  // leaf
        const int g = ~cn;
        if (g == f) continue;
        const int tg = ftag ? ftag[g] : -1;
        if (query_all ? (g < f) : (tg >= 0 && g < f)) continue;
        const int4 cv = F[g];
        const int ci[3] = {cv.x, cv.y, cv.z};
        const float4 a = pos[cv.x], b = pos[cv.y], cc = pos[cv.z];
        const float3 C[3] = {make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z),
                             make_float3(cc.x, cc.y, cc.z)};
        if (exact::faces_intersect(T, ti, fiT, C, ci, unpack_info(info[g]))) {
          if (undo) {
            if (tf >= 0) undo[tf] = 1;
            if (tg >= 0) undo[tg] = 1;
          }
          const int slot = atomicAdd(&dc->n_pairs, 1);
          if (pairs_out && slot < cap) {
            pairs_out[2 * slot] = min(f, g);
            pairs_out[2 * slot + 1] = max(f, g);
          }
        }
      } else if (next < 0) {
        next = cn;
      } else {
        if (sp >= kStack) {
          atomicOr(&dc->overflow, 1);
          return;
        }
        stack[sp++] = cn;
      }
    }
    if (next >= 0) {
      node = next;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
}

// ---- split check: traversal -> candidate pairs -> exact pair test --------
// Candidates are bucketed by the number of shared vertex indices (0, 1, >=2)
// so that warps of the pair kernel follow one branch of the predicate.
struct CandBufs {
  int2* c[3];
  int64_t cap[3];
};

// Appends candidate pair (f, g) to the bucket of its shared-vertex count
// (warp-aggregated over the lanes that append in the same call)
__device__ __forceinline__ void append_candidate(int f, const int4& tv, int g,
                                                 const int4* __restrict__ F, CandBufs& cb,
                                                 int* __restrict__ ncand) {
  const int4 gv = F[g];
  int s = 0;
  s += (gv.x == tv.x) | (gv.x == tv.y) | (gv.x == tv.z);
  s += (gv.y == tv.x) | (gv.y == tv.y) | (gv.y == tv.z);
  s += (gv.z == tv.x) | (gv.z == tv.y) | (gv.z == tv.z);
  const int r = s >= 2 ? 2 : s;
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, r);
  const int leader = __ffs(peers) - 1;
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == leader) base = atomicAdd(&ncand[r], __popc(peers));
  base = __shfl_sync(peers, base, leader);
  const int slot = base + __popc(peers & ((1u << lane) - 1u));
  if (slot < cb.cap[r]) cb.c[r][slot] = make_int2(f, g);
}

// Depth-first traversal of the subtree at `node` for query f (one thread),
// two nodes per step: the two deepest pending nodes are loaded together, so a
// lane has two node loads in flight instead of one chain.  Children are pushed
// shallower node first, so the stack stays sorted by depth and holds at most
// two nodes per level (a visited pair leaves at most two of its up to four
// children behind): 2 x 62 levels fit in kStackPair entries.
// Returns false after a stack or visit-cap overflow (flagged in dc).
constexpr int kStackPair = 128;
__device__ __forceinline__ bool dfs_query(const float* __restrict__ nodes, int node, int n, int f,
                                          const int4& tv, const float3& lo, const float3& hi,
                                          const int32_t* __restrict__ ftag, int query_all,
                                          const int4* __restrict__ F, CandBufs& cb,
                                          int* __restrict__ ncand, RoundCounters* __restrict__ dc) {
  int stack[kStackPair];
  int sp = 0;
  int a = node, b = -1;  // the pair visited next (b < 0: a alone)
  for (int visits = 0;; visits += 2) {
    if (visits >= 2 * n) {
      atomicOr(&dc->overflow, 4);
      return false;
    }
    const NodeHits ha = visit(nodes, a, lo, hi);
    NodeHits hb = visit(nodes, b >= 0 ? b : a, lo, hi);
    if (b < 0) hb.l = hb.r = false;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const NodeHits& h = k < 2 ? ha : hb;
      if (!((k & 1) ? h.r : h.l)) continue;
      const int cn = (k & 1) ? h.R : h.L;
      if (cn < 0) {
        const int g = ~cn;
        if (g == f) continue;
        const int tg = ftag ? ftag[g] : -1;
        if (query_all ? (g < f) : (tg >= 0 && g < f)) continue;
        append_candidate(f, tv, g, F, cb, ncand);
      } else {
        if (sp >= kStackPair) {
          atomicOr(&dc->overflow, 1);
          return false;
        }
        stack[sp++] = cn;
      }
    }
    if (sp == 0) return true;
    b = stack[--sp];
    a = sp > 0 ? stack[--sp] : -1;
    if (a < 0) {
      a = b;
      b = -1;
    }
  }
}

// One thread per query face while there are many queries; when there are at
// most two per warp (the small late rounds, where a query's chain of
// dependent node loads is the kernel's time), one warp per query: the warp
// expands the tree breadth-first over its lanes until the frontier fills
// them, then each lane finishes its frontier nodes depth-first, so the chain
// is about the tree's depth instead of one load per overlapping node.
__global__ void __launch_bounds__(kBlock) k_traverse(
    const float* __restrict__ nodes, const int* n_dev, int n_host, const float4* __restrict__ pos,
    const int4* __restrict__ F, const uint8_t* __restrict__ fdead,
    const int32_t* __restrict__ ftag, int query_all, const int32_t* __restrict__ qlist,
    const int* __restrict__ qcount, CandBufs cb, int* __restrict__ ncand,
    RoundCounters* __restrict__ dc, const int32_t* __restrict__ vmesh,
    const int32_t* __restrict__ mroot) {
  __shared__ int frontier[kBlock / 32][64];
  const int n = dev_n(n_dev, n_host);
  const int total = query_all ? n : *qcount;
  if (n < 2) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  if ((int64_t)total > 2 * warps) {  // block-uniform: one thread per query
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
      const int f = query_all ? i : qlist[i];
      if (fdead && fdead[f]) continue;
      const int tf = ftag ? ftag[f] : -1;
      if (!query_all && tf < 0) continue;
      const int4 tv = F[f];
      const float4 a = pos[tv.x], b = pos[tv.y], c = pos[tv.z];
      const float3 lo = make_float3(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y),
                                    fminf(fminf(a.z, b.z), c.z));
      const float3 hi = make_float3(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y),
                                    fmaxf(fmaxf(a.z, b.z), c.z));
      dfs_query(nodes, mroot ? mroot[vmesh[tv.x]] : 0, n, f, tv, lo, hi, ftag, query_all, F, cb,
                ncand, dc);
    }
    return;
  }
  int* fr = frontier[threadIdx.x >> 5];
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t i = w0; i < total; i += warps) {  // warp-uniform
    const int f = query_all ? (int)i : qlist[i];
    if (fdead && fdead[f]) continue;
    if (!query_all && (ftag ? ftag[f] : -1) < 0) continue;
    const int4 tv = F[f];
    const float4 a = pos[tv.x], b = pos[tv.y], c = pos[tv.z];
    const float3 lo = make_float3(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y),
                                  fminf(fminf(a.z, b.z), c.z));
    const float3 hi = make_float3(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y),
                                  fmaxf(fmaxf(a.z, b.z), c.z));
    if (lane == 0) fr[0] = mroot ? mroot[vmesh[tv.x]] : 0;
    int nf = 1;
    __syncwarp();
    // breadth-first while the frontier is narrower than the warp (at most 62
    // entries after a step)
    for (int level = 0; nf > 0 && nf < 32 && level < kStack; level++) {
      int kids[2] = {-1, -1}, nk = 0;
      if (lane < nf) {
        const NodeHits h = visit(nodes, fr[lane], lo, hi);
#pragma unroll
        for (int k = 0; k < 2; k++) {
          if (!(k ? h.r : h.l)) continue;
          const int cn = k ? h.R : h.L;
          if (cn < 0) {
            const int g = ~cn;
            if (g == f) continue;
            const int tg = ftag ? ftag[g] : -1;
            if (query_all ? (g < f) : (tg >= 0 && g < f)) continue;
            append_candidate(f, tv, g, F, cb, ncand);
          } else {
            kids[nk++] = cn;
          }
        }
      }
      int incl = nk;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      __syncwarp();  // every lane has read its frontier entry
      const int o = incl - nk;
      for (int k = 0; k < nk; k++) fr[o + k] = kids[k];
      nf = __shfl_sync(0xffffffffu, incl, 31);
      __syncwarp();
    }
    // depth-first from the frontier nodes, one per lane (two at most)
    for (int j = lane; j < nf; j += 32)
      dfs_query(nodes, fr[j], n, f, tv, lo, hi, ftag, query_all, F, cb, ncand, dc);
    __syncwarp();  // the next query overwrites the frontier
  }
}

// The re-check after an undo.  The previous mesh M_1 is intersection-free, so
// a restored face (an M_1 face again) meets no unchanged or restored face, and
// faces of standing collapses met no other in the last iteration (both
// collapses would have been undone); every intersecting pair of this
// iteration is therefore a restored face and a live face of a standing
// collapse (ftag >= 0), found from the restored side.  The tree is the one
// refitted for the first iteration: the standing faces have not moved since,
// so their leaf boxes, and every ancestor's, still contain them (the stale
// leaves of restored faces only add candidates that the tag test drops).
// Each query also rewrites its face's predicate info for the pair test.
__global__ void __launch_bounds__(kBlock) k_traverse_restored(
    const float* __restrict__ nodes, const int* n_dev, const float4* __restrict__ pos,
    const int4* __restrict__ F, const uint8_t* __restrict__ fdead,
    const int32_t* __restrict__ ftag, const int32_t* __restrict__ rlist, CandBufs cb,
    int* __restrict__ ncand, RoundCounters* __restrict__ dc, uint8_t* __restrict__ info,
    const int32_t* __restrict__ vmesh, const int32_t* __restrict__ mroot) {
  const int n = *n_dev;
  const int lo = dc->rest_lo, hi = dc->rest_mid;
  if (n < 2) return;
  for (int i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x) {
    const int f = rlist[i];
    const int4 tv = F[f];
    const float4 a = pos[tv.x], b = pos[tv.y], c = pos[tv.z];
    info[f] = pack_info(exact::face_info(make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z),
                                         make_float3(c.x, c.y, c.z)));
    const float3 qlo = make_float3(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y),
                                   fminf(fminf(a.z, b.z), c.z));
    const float3 qhi = make_float3(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y),
                                   fmaxf(fmaxf(a.z, b.z), c.z));
    int stack[kStack];
    int sp = 0, node = mroot ? mroot[vmesh[tv.x]] : 0;  // the query's own mesh
    for (int visits = 0;; visits++) {
      if (visits >= 2 * n) {
        atomicOr(&dc->overflow, 4);
        break;
      }
      const NodeHits h = visit(nodes, node, qlo, qhi);
      int next = -1;
#pragma unroll
      for (int k = 0; k < 2; k++) {
        if (!(k ? h.r : h.l)) continue;
        const int cn = k ? h.R : h.L;
        if (cn < 0) {
          const int g = ~cn;
          if (g == f || ftag[g] < 0 || fdead[g]) continue;
          const int4 gv = F[g];
          int s = 0;
          s += (gv.x == tv.x) | (gv.x == tv.y) | (gv.x == tv.z);
          s += (gv.y == tv.x) | (gv.y == tv.y) | (gv.y == tv.z);
          s += (gv.z == tv.x) | (gv.z == tv.y) | (gv.z == tv.z);
          const int r = s >= 2 ? 2 : s;
          // warp-aggregated append into bucket r
          const unsigned act = __activemask();
          const unsigned peers = __match_any_sync(act, r);
          const int leader = __ffs(peers) - 1;
          const int lane = threadIdx.x & 31;
          int base = 0;
          if (lane == leader) base = atomicAdd(&ncand[r], __popc(peers));
          base = __shfl_sync(peers, base, leader);
          const int slot = base + __popc(peers & ((1u << lane) - 1u));
          if (slot < cb.cap[r]) cb.c[r][slot] = make_int2(f, g);
        } else if (next < 0) {
          next = cn;
        } else {
          if (sp >= kStack) {
            atomicOr(&dc->overflow, 1);
            next = -2;
            break;
          }
          stack[sp++] = cn;
        }
      }
      if (next == -2) break;
      if (next >= 0) {
        node = next;
      } else {
        if (sp == 0) break;
        node = stack[--sp];
      }
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_pairs(
    CandBufs cb, const int* __restrict__ ncand, const float4* __restrict__ pos,
    const int4* __restrict__ F, const uint8_t* __restrict__ info,
    const int32_t* __restrict__ ftag, uint8_t* __restrict__ undo, RoundCounters* __restrict__ dc,
    uint32_t* __restrict__ vgap) {
  const int n2 = min((int64_t)ncand[2], cb.cap[2]);
  const int n1 = min((int64_t)ncand[1], cb.cap[1]);
  const int n0 = min((int64_t)ncand[0], cb.cap[0]);
  const int total = n2 + n1 + n0;
  if (blockIdx.x == 0 && threadIdx.x == 0 &&
      (ncand[0] > cb.cap[0] || ncand[1] > cb.cap[1] || ncand[2] > cb.cap[2]))
    dc->cand_overflow = 1;
  int found = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int2 p = i < n2 ? cb.c[2][i] : (i < n2 + n1 ? cb.c[1][i - n2] : cb.c[0][i - n2 - n1]);
    const int f = p.x, g = p.y;
    const int4 tv = F[f], cv = F[g];
    if (vgap && i >= n2 + n1) {
      // boxes of faces with no common vertex overlap: each face's corners get
      // the distance of the other face's centroid to its plane (a clearance
      // estimate for the learned proposal; positive floats order as integers)
      const float4 a0 = pos[tv.x], a1 = pos[tv.y], a2 = pos[tv.z];
      const float4 b0 = pos[cv.x], b1 = pos[cv.y], b2 = pos[cv.z];
      const float3 na = cross3f(sub3f(a1, a0), sub3f(a2, a0));
      const float3 nb = cross3f(sub3f(b1, b0), sub3f(b2, b0));
      const float3 ca = make_float3((a0.x + a1.x + a2.x) / 3.f, (a0.y + a1.y + a2.y) / 3.f,
                                    (a0.z + a1.z + a2.z) / 3.f);
      const float3 cb = make_float3((b0.x + b1.x + b2.x) / 3.f, (b0.y + b1.y + b2.y) / 3.f,
                                    (b0.z + b1.z + b2.z) / 3.f);
      const float la = sqrtf(na.x * na.x + na.y * na.y + na.z * na.z);
      const float lb = sqrtf(nb.x * nb.x + nb.y * nb.y + nb.z * nb.z);
      const float da = la > 0.f ? fabsf(na.x * (cb.x - a0.x) + na.y * (cb.y - a0.y) +
                                        na.z * (cb.z - a0.z)) / la : 0.f;
      const float db = lb > 0.f ? fabsf(nb.x * (ca.x - b0.x) + nb.y * (ca.y - b0.y) +
                                        nb.z * (ca.z - b0.z)) / lb : 0.f;
      const unsigned ua = __float_as_uint(da), ub = __float_as_uint(db);
      atomicMin(&vgap[tv.x], ua); atomicMin(&vgap[tv.y], ua); atomicMin(&vgap[tv.z], ua);
      atomicMin(&vgap[cv.x], ub); atomicMin(&vgap[cv.y], ub); atomicMin(&vgap[cv.z], ub);
    }
    const int ti[3] = {tv.x, tv.y, tv.z};
    const int ci[3] = {cv.x, cv.y, cv.z};
    float3 T[3], C[3];
    {
      const float4 a = pos[tv.x], b = pos[tv.y], c = pos[tv.z];
      T[0] = make_float3(a.x, a.y, a.z);
      T[1] = make_float3(b.x, b.y, b.z);
      T[2] = make_float3(c.x, c.y, c.z);
      const float4 d = pos[cv.x], e = pos[cv.y], h = pos[cv.z];
      C[0] = make_float3(d.x, d.y, d.z);
      C[1] = make_float3(e.x, e.y, e.z);
      C[2] = make_float3(h.x, h.y, h.z);
    }
    if (exact::faces_intersect(T, ti, unpack_info(info[f]), C, ci, unpack_info(info[g]))) {
      found++;
      if (undo) {
        const int tf = ftag[f], tg = ftag[g];
        if (tf >= 0) undo[tf] = 1;
        if (tg >= 0) undo[tg] = 1;
      }
    }
  }
  found = __reduce_add_sync(0xffffffffu, found);
  if ((threadIdx.x & 31) == 0 && found) atomicAdd(&dc->n_pairs, found);
}

__global__ void k_tri_batch(const float* __restrict__ P, const int32_t* __restrict__ idx,
                            int64_t n, uint8_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* p = P + 18 * i;
  float3 T[3], C[3];
  for (int k = 0; k < 3; k++) {
    T[k] = make_float3(p[3 * k], p[3 * k + 1], p[3 * k + 2]);
    C[k] = make_float3(p[9 + 3 * k], p[9 + 3 * k + 1], p[9 + 3 * k + 2]);
  }
  const int ti[3] = {idx[6 * i], idx[6 * i + 1], idx[6 * i + 2]};
  const int ci[3] = {idx[6 * i + 3], idx[6 * i + 4], idx[6 * i + 5]};
  out[i] = exact::faces_intersect(T, ti, exact::face_info(T[0], T[1], T[2]), C, ci,
                                  exact::face_info(C[0], C[1], C[2]))
               ? 1
               : 0;
}

__global__ void k_orient3d_batch(const float* __restrict__ P, int64_t n, int8_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* p = P + 12 * i;
  out[i] = (int8_t)exact::orient3d(make_float3(p[0], p[1], p[2]), make_float3(p[3], p[4], p[5]),
                                   make_float3(p[6], p[7], p[8]), make_float3(p[9], p[10], p[11]));
}

__global__ void k_orient2d_batch(const float* __restrict__ P, int64_t n, int8_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* p = P + 6 * i;
  out[i] = (int8_t)exact::orient2d(p[0], p[1], p[2], p[3], p[4], p[5]);
}

}  // namespace

// Buffers for trees of up to n_max faces (nothing is allocated later, so a
// build can be captured in a graph).
pamo_status bvh_alloc(Bvh& b, int n_max, cudaStream_t st) {
  size_t nb, pb, fb, kvb, hb, ab;
  int64_t hw;
  bvh_bytes(n_max, &nb, &pb, &fb, &kvb, &hb, &ab, &hw);
  PAMO_TRY(buf_reserve(b.nodes, nb, st));
  PAMO_TRY(buf_reserve(b.parent, pb, st));
  PAMO_TRY(buf_reserve(b.flags, fb, st));
  PAMO_TRY(buf_reserve(b.keys, kvb, st));
  PAMO_TRY(buf_reserve(b.vals, kvb, st));
  PAMO_TRY(buf_reserve(b.keys2, kvb, st));
  PAMO_TRY(buf_reserve(b.vals2, kvb, st));
  PAMO_TRY(buf_reserve(b.hist, hb, st));
  PAMO_TRY(buf_reserve(b.face_aux, ab, st));
  PAMO_TRY(buf_reserve(b.sort_len, 16, st));
  PAMO_TRY(buf_reserve(b.posn, sizeof(int32_t) * ((size_t)n_max + 1), st));
  PAMO_TRY(buf_reserve(b.sums, sizeof(int32_t) * scan_sums_count(hw > n_max ? hw : n_max), st));
  if (b.n_mesh > 1) {
    PAMO_TRY(buf_reserve(b.hkeys, kvb, st));
    PAMO_TRY(buf_reserve(b.hkeys2, kvb, st));
    PAMO_TRY(buf_reserve(b.mroot, sizeof(int32_t) * (size_t)b.n_mesh, st));
  }
  b.n_max = n_max;
  return PAMO_OK;
}

void bvh_bytes(int n, size_t* nodes, size_t* parent, size_t* flags, size_t* kv, size_t* hist,
               size_t* aux, int64_t* hist_words) {
  const int tiles = n > 0 ? (n + kSortTile - 1) / kSortTile : 1;
  // 64-byte internal nodes, then 32-byte leaf boxes (read by the refit)
  *nodes = sizeof(float) * (16 * (size_t)(n > 1 ? n : 1) + 8 * (size_t)(n > 1 ? n : 1));
  *parent = sizeof(int32_t) * (size_t)(2 * n + 1);
  *flags = sizeof(int32_t) * (size_t)(n + 2);
  *kv = sizeof(uint32_t) * (size_t)(n > 1 ? n : 1);
  *hist = sizeof(int32_t) * (size_t)(2 * 256 * tiles + 2);
  *aux = (size_t)n + 16;
  *hist_words = 256 * (int64_t)tiles;
}

// Build over faces [0, n) (n from n_dev when set, else n_host) in the
// preallocated buffers of b.  carry = true keeps the current leaf order and
// keys (see bvh_compact_order) and only rebuilds the hierarchy.
pamo_status bvh_build(Bvh& b, const float4* pos, const int4* F, const uint8_t* fdead,
                      const int* n_dev, int n_host, const float lo[3], const float hi[3],
                      bool carry, int grid, cudaStream_t st) {
  unsigned* keys = (unsigned*)b.keys.p;
  int32_t* vals = (int32_t*)b.vals.p;
  unsigned* hk = b.n_mesh > 1 ? (unsigned*)b.hkeys.p : nullptr;
  if (!carry) {
    float inv[3];
    for (int k = 0; k < 3; k++) {
      float e = hi[k] - lo[k];
      inv[k] = e > 0.f ? 1.0f / e : 0.0f;
    }
    unsigned* keys2 = (unsigned*)b.keys2.p;
    int32_t* vals2 = (int32_t*)b.vals2.p;
    unsigned* hk2 = hk ? (unsigned*)b.hkeys2.p : nullptr;
    static const int g_keys = occ_grid(k_leaf_keys);
    k_leaf_keys<<<g_keys, kBlock, 0, st>>>(pos, F, fdead, n_dev, n_host, lo[0], lo[1], lo[2],
                                           inv[0], inv[1], inv[2], hk ? b.vmesh : nullptr,
                                           b.mframe, keys, hk, vals); note_launch();
    const int tiles_max = (b.n_max + kSortTile - 1) / kSortTile;
    int32_t* hist = (int32_t*)b.hist.p;
    int32_t* offs = hist + 256 * (tiles_max > 0 ? tiles_max : 1) + 1;
    int* len = (int*)b.sort_len.p;
    k_sort_len<<<1, 1, 0, st>>>(n_dev, n_host, len); note_launch();
    // LSD: the four bytes of the Morton word, then the bytes of the mesh id
    int hi_passes = 0;
    for (int m = b.n_mesh - 1; m > 0; m >>= 8) hi_passes++;
    for (int pass = 0; pass < 4 + hi_passes; pass++) {
      const bool from_hi = pass >= 4;
      const int shift = 8 * (from_hi ? pass - 4 : pass);
      k_digit_hist<<<grid, kBlock, 0, st>>>(from_hi ? hk : keys, n_dev, n_host, shift, hist); note_launch();
      PAMO_TRY(scan_dev_i32(hist, len, offs, (int32_t*)b.sums.p, grid, st));
      k_digit_scatter<<<grid, kBlock, 0, st>>>(keys, vals, hk, from_hi ? 1 : 0, n_dev, n_host,
                                               shift, offs, keys2, vals2, hk2); note_launch();
      PAMO_CUDA(cudaGetLastError());
      std::swap(keys, keys2);
      std::swap(vals, vals2);
      std::swap(hk, hk2);
    }
    if (keys != (unsigned*)b.keys.p) {  // an odd number of passes: back to the primary buffers
      k_copy_order<<<grid, kBlock, 0, st>>>(vals, keys, hk, n_dev, n_host, vals2, keys2, hk2); note_launch();
      keys = keys2;
      vals = vals2;
      hk = hk2;
    }
  }
  static const int g_karras = occ_grid(k_karras);
  k_karras<<<g_karras, kBlock, 0, st>>>(keys, hk, vals, n_dev, n_host, (float*)b.nodes.p,
                                        (int32_t*)b.parent.p, (int32_t*)b.mroot.p); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return bvh_refit(b, pos, F, fdead, n_dev, n_host, grid, st);
}

pamo_status bvh_refit(Bvh& b, const float4* pos, const int4* F, const uint8_t* fdead,
                      const int* n_dev, int n_host, int grid, cudaStream_t st) {
  int32_t* fl = (int32_t*)b.flags.p;
  PAMO_CUDA(cudaMemsetAsync(fl, 0, sizeof(int32_t) * (size_t)(b.n_max + 2), st));
  float4* lbox = reinterpret_cast<float4*>((float*)b.nodes.p + 16 * (size_t)(b.n_max > 1 ? b.n_max : 1));
  static const int g_leaf = occ_grid(k_leaf_boxes);
  k_leaf_boxes<<<g_leaf, kBlock, 0, st>>>(pos, F, fdead, (const int32_t*)b.vals.p, n_dev, n_host,
                                          lbox, (uint8_t*)b.face_aux.p); note_launch();
  static const int g_refit = occ_grid(k_refit_nodes);
  k_refit_nodes<<<g_refit, kBlock, 0, st>>>(lbox, n_dev, n_host, (float*)b.nodes.p,
                                            (const int32_t*)b.parent.p, fl, fl + b.n_max + 1); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status bvh_check(Bvh& b, const float4* pos, const int4* F, const uint8_t* fdead,
                      const int32_t* ftag, int query_all, const int32_t* qlist,
                      const int* qcount, int64_t nq_max, uint8_t* undo, RoundCounters* dc,
                      int32_t* pairs_out, int64_t cap, int n_host, cudaStream_t st) {
  // fold a refit overflow into the round's overflow word
  k_fold_overflow<<<1, 1, 0, st>>>((const int32_t*)b.flags.p + b.n_max + 1, &dc->overflow); note_launch();
  const int64_t threads = query_all ? n_host : nq_max;
  const bool many = b.n_mesh > 1;
  k_query<<<grid_for(threads), kBlock, 0, st>>>((const float*)b.nodes.p, nullptr, n_host, pos, F,
                                                fdead, (const uint8_t*)b.face_aux.p, ftag,
                                                query_all, qlist, qcount, undo, dc, pairs_out,
                                                cap, many ? b.vmesh : nullptr,
                                                many ? (const int32_t*)b.mroot.p : nullptr); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status bvh_compact_order(Bvh& b, const uint8_t* fdead, const int32_t* dead_before,
                              const int* n_old_dev, const int* n_new_dev, int grid,
                              cudaStream_t st) {
  // runs on every check outcome (sizes 0 when the round does not commit), so
  // it must leave the tree intact: the positions of the live leaves are in
  // their own buffer (posn, scanned by the caller)
  const int32_t* posn = (const int32_t*)b.posn.p;
  const bool many = b.n_mesh > 1;
  k_order_write<<<grid, kBlock, 0, st>>>((const int32_t*)b.vals.p, (const unsigned*)b.keys.p,
                                         many ? (const unsigned*)b.hkeys.p : nullptr, n_old_dev,
                                         fdead, posn, dead_before, (int32_t*)b.vals2.p,
                                         (unsigned*)b.keys2.p,
                                         many ? (unsigned*)b.hkeys2.p : nullptr); note_launch();
  k_copy_order<<<grid, kBlock, 0, st>>>((const int32_t*)b.vals2.p, (const unsigned*)b.keys2.p,
                                        many ? (const unsigned*)b.hkeys2.p : nullptr, n_new_dev, 0,
                                        (int32_t*)b.vals.p, (unsigned*)b.keys.p,
                                        many ? (unsigned*)b.hkeys.p : nullptr); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status bvh_check_split(Bvh& b, const float4* pos, const int4* F, const uint8_t* fdead,
                            const int32_t* ftag, int query_all, const int32_t* qlist,
                            const int* qcount, uint8_t* undo, RoundCounters* dc, int2* const cand[3],
                            const int64_t cap[3], int* ncand, const int* n_dev, int grid,
                            cudaStream_t st) {
  k_check_begin<<<1, 1, 0, st>>>((const int32_t*)b.flags.p + b.n_max + 1, dc, 0); note_launch();
  CandBufs cb;
  for (int r = 0; r < 3; r++) {
    cb.c[r] = cand[r];
    cb.cap[r] = cap[r];
  }
  const bool many = b.n_mesh > 1;
  static const int g_trav = occ_grid(k_traverse);
  static const int g_pairs = occ_grid(k_pairs, kItemBlock);
  k_traverse<<<g_trav, kBlock, 0, st>>>((const float*)b.nodes.p, n_dev, 0, pos, F, fdead, ftag,
                                        query_all, qlist, qcount, cb, ncand, dc,
                                        many ? b.vmesh : nullptr,
                                        many ? (const int32_t*)b.mroot.p : nullptr); note_launch();
  k_pairs<<<g_pairs, kItemBlock, 0, st>>>(cb, ncand, pos, F, (const uint8_t*)b.face_aux.p, ftag, undo,
                                   dc, b.vgap); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status bvh_recheck_restored(Bvh& b, const float4* pos, const int4* F, const uint8_t* fdead,
                                 const int32_t* ftag, const int32_t* rlist, uint8_t* undo,
                                 RoundCounters* dc, int2* const cand[3], const int64_t cap[3],
                                 int* ncand, const int* n_dev, cudaStream_t st) {
  k_check_begin<<<1, 1, 0, st>>>((const int32_t*)b.flags.p + b.n_max + 1, dc, 1); note_launch();
  CandBufs cb;
  for (int r = 0; r < 3; r++) {
    cb.c[r] = cand[r];
    cb.cap[r] = cap[r];
  }
  const bool many = b.n_mesh > 1;
  static const int g_trav = occ_grid(k_traverse_restored);
  static const int g_pairs = occ_grid(k_pairs, kItemBlock);
  k_traverse_restored<<<g_trav, kBlock, 0, st>>>((const float*)b.nodes.p, n_dev, pos, F, fdead,
                                                 ftag, rlist, cb, ncand, dc,
                                                 (uint8_t*)b.face_aux.p,
                                                 many ? b.vmesh : nullptr,
                                                 many ? (const int32_t*)b.mroot.p : nullptr); note_launch();
  k_pairs<<<g_pairs, kItemBlock, 0, st>>>(cb, ncand, pos, F, (const uint8_t*)b.face_aux.p, ftag,
                                          undo, dc, b.vgap); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

void bvh_free(Bvh& b, cudaStream_t st) {
  buf_free(b.nodes, st);
  buf_free(b.parent, st);
  buf_free(b.flags, st);
  buf_free(b.keys, st);
  buf_free(b.vals, st);
  buf_free(b.keys2, st);
  buf_free(b.vals2, st);
  buf_free(b.hist, st);
  buf_free(b.face_aux, st);
  buf_free(b.sort_len, st);
  buf_free(b.sums, st);
  buf_free(b.posn, st);
  buf_free(b.hkeys, st);
  buf_free(b.hkeys2, st);
  buf_free(b.mroot, st);
}

pamo_status tri_batch(const float* P, const int32_t* idx, int64_t n, uint8_t* out,
                      cudaStream_t st) {
  if (n <= 0) return PAMO_OK;
  k_tri_batch<<<grid_for(n), kBlock, 0, st>>>(P, idx, n, out); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status orient3d_batch(const float* P, int64_t n, int8_t* out, cudaStream_t st) {
  if (n <= 0) return PAMO_OK;
  k_orient3d_batch<<<grid_for(n), kBlock, 0, st>>>(P, n, out); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status orient2d_batch(const float* P, int64_t n, int8_t* out, cudaStream_t st) {
  if (n <= 0) return PAMO_OK;
  k_orient2d_batch<<<grid_for(n), kBlock, 0, st>>>(P, n, out); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // namespace pamo
