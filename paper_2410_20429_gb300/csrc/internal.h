// internal.h -- device data layout and launch wrappers shared by the CUDA
// translation units of libmars (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mars.h"

namespace mars {

constexpr int NT = MARS_NUM_SLOTS;
constexpr int NSTAT = MARS_NUM_STATS;
constexpr int GUIDE_BINS = MARS_GUIDE_BINS;
constexpr int MAXD = MARS_MAX_DEPTH;
constexpr uint32_t DIM_ROUND = 96;   // Philox dimension of the Alg. 1 draw
constexpr uint32_t DIM_CAMERA = 97;  // Philox dimension of the pixel jitter
// Philox dimension of step k of the light subpath of light connection sample
// s: DIM_LIGHT + 8 s + k (k = 0 light and point, 1 emission direction, k >= 2
// the bounce at surface vertex k - 1 and its Russian roulette)
constexpr uint32_t DIM_LIGHT = 128;
constexpr int LIGHT_MAX = MARS_LIGHT_MAX;

// ---------------------------------------------------------------- scene
// Primitive record: four float4 per primitive.
//   w-bits of p[0]: (material << 2) | type   (type 0 quad, 1 sphere, 2 triangle)
//   quad:     p0 | e1 | e2 | unit normal, w = light index (int bits, -1 if none)
//   sphere:   centre | (r, 1/r, 0, 0) | - | -
//   triangle: v0 | e1 = v1 - v0 | e2 = v2 - v0 | unit normal
enum { PRIM_QUAD = 0, PRIM_SPHERE = 1, PRIM_TRI = 2 };

// BVH node (Karras 2012 binary LBVH): the bounds of both children live in the
// parent so one 64-byte fetch tests two boxes.
//   a = (left lo xyz,  left child)   b = (left hi xyz,  right child)
//   c = (right lo xyz, 0)            d = (right hi xyz, 0)
// child >= 0: internal node index; child < 0: leaf holding primitive ~child.
struct BvhNode {
  float4 a, b, c, d;
};

// 4-wide BVH node (collapsed from the binary LBVH on the host): the boxes of up
// to four children as structure of arrays, one float4 per coordinate, and the
// children: >= 0 internal node, < 0 primitive ~child, BVH4_EMPTY unused.
constexpr int BVH4_EMPTY = 0x7fffffff;
struct Bvh4Node {
  float4 lox, loy, loz, hix, hiy, hiz;
  int4 child;
  float4 pad;
};

// Material: m0 = (type, alpha, reflective, emissive), m1 = (colour rgb, 0),
// m2 = (emitted radiance rgb, 0).
// Light: l0 = (p0 xyz, cdf), l1 = (e1 xyz, pmf), l2 = (e2 xyz, area),
//        l3 = (unit normal xyz, primitive index bits), l4 = (radiance rgb, 0).
struct DevScene {
  const float4* prims;
  const BvhNode* nodes;
  const Bvh4Node* nodes4;
  int n_nodes4;
  const float4* mats;
  const float4* lights;
  int n_prims, n_quads, n_lights, n_mats;
  float lo[3], ext[3];
  float eps;
  float cam_o[3], cam_f[3], cam_r[3], cam_u[3];
  float tanh_half, aspect;
  int width, height;
};

// ---------------------------------------------------------------- arena
// One arena for all depth waves of a tile; wave d occupies
// [base[d], base[d] + count[d]).  Structure of arrays, one float4 (or float2)
// per field group so every load/store is a coalesced 8- or 16-byte access.
//   R0 = (origin xyz, pixel)            R1 = (direction xyz, A = beta_t p_t)
//   R2 = (T at the hit xyz, S_ind)      R3 = (f|cos|/p xyz, NEE weight factor)
//   R4 = (lineage lo, lineage hi, parent cell, 1 / sum beta_k p_k)
//   H  = (t, primitive: -1 missed, -2 not traced) from the trace kernel; the
//        shade kernel then overwrites it with (first child, first shadow ray)
//        as slot indices, the first two addresses the reverse pass needs
//   V0 = (E xyz, flags)                 V1 = (G xyz, -)
//   V2 = (clamp limit xyz, cell)        V3 = (beta BSDF, NEE, guided, -)
//   V4 = (Le luminance, 1/S_beta, parent cell, bin)
//   S  = (sample value xyz, cost)
// NEE shadow rays of wave d occupy [sbase[d], sbase[d] + scount[d]) of a second
// arena: SH0 = (origin xyz, tmax; < 0: nothing to trace), SH1 = (direction, -),
// SH2 = (sample value if visible, -), zeroed by the shadow kernel when occluded.
// Only samples with a nonzero value need a ray: their slots are listed in
// SL[sbase[d], sbase[d] + slcount[d]) (a compacted work list), and SH0/SH1 are
// written for them alone.
//
// With light connections (MARS_TECH_LIGHT) a ray carries the running sums of
// the whole-path weights instead of the guided technique's fields:
//   R2.w = |cos| at the parent of the ray's direction (instead of S_ind),
//   R4.zw, R5 = Z[1..6]: Z[1] = the parent's light connection count, Z[l] the
//   term of a light connection l vertices back, relative to the camera prefix
//   up to the parent (divided by the last step's density at the hit),
// V3.w holds the first light connection slot of the vertex, and the light
// connection samples of wave d occupy [lbase[d], lbase[d] + lcount[d]) of a
// third region: LJ0..LJ7 the camera vertex's context (written by the shade
// kernel), LR = (first light vertex slot, light vertex count m, pN, cost)
// written by the light-subpath kernel.  The light vertices of wave d's samples
// occupy [vbase(d), vbase(d) + vcount[d]) of a fourth region, vbase(d) the sum
// of the earlier waves' vcount, each sample's m vertices in order:
//   LV0 = (position, primitive), LV1 = (unit direction to the previous light
//   vertex, distance to it), LV2 = (throughput alpha, area density lambda),
//   LV3 = (geometric normal, cell), LV4 = (reverse f cos towards the previous
//   vertex with the next one outgoing, its density), LV5 = (|cos| at the
//   previous vertex towards this one, sample slot, index in the subpath, -),
// and LC = (weighted contribution of the connection to it if visible, -),
// written by the connection kernel.
constexpr int NR = 5, NV = 5, NSH = 3, NLJ = 8, NLV = 6;
constexpr int SLOT_BYTES = (NR + NV + 1) * 16 + 8 + 4;  // per ray slot
constexpr int SHADOW_BYTES = NSH * 16 + 4;          // per shadow-ray slot
// R5 per ray slot, LJ and LR per connection slot, LV and LC per light vertex
// slot (as many of each as ray slots)
constexpr int LIGHT_SLOT_BYTES = 16 + (NLJ + 1) * 16 + (NLV + 1) * 16;
struct Arena {
  float4* R[NR];
  float2* H;
  float4* V[NV];
  float4* S;
  float* M;   // path multiplicity of the ray (product of the budgets that drew its path)
  float4* SH[NSH];
  unsigned int* SL;
  float4* R5;        // light connections only
  float4* LJ[NLJ];
  float4* LR;
  float4* LV[NLV];
  float4* LC;
  uint64_t cap;   // ray slots
  uint64_t scap;  // shadow-ray slots
  uint64_t lcap;  // light connection slots (0 without light connections)
  uint64_t vcap;  // light vertex slots (0 without light connections)
};

// V0.w flag bits
constexpr uint32_t F_TRACED = 1u << 24;
constexpr uint32_t F_EST = 1u << 25;

// the image pass's block sums go to IMG_SLOTS addresses (block b adds to slot
// b mod IMG_SLOTS) instead of one: same-address float64 atomics from every block
// of the grid serialise
constexpr int IMG_SLOTS = 32;

// Device-resident per-iteration counters.
struct DevCounters {
  unsigned long long base[MAXD + 2];
  unsigned long long count[MAXD + 2];
  unsigned long long sbase[MAXD + 2];   // shadow rays of wave d
  unsigned long long scount[MAXD + 2];
  unsigned long long slcount[MAXD + 2];  // shadow rays of wave d that need tracing
  unsigned long long lbase[MAXD + 2];    // light connection samples of wave d
  unsigned long long lcount[MAXD + 2];
  unsigned long long vcount[MAXD + 2];   // light subpath vertices of wave d's samples
  unsigned long long light_rays, conn_rays;  // light-subpath closest hits, connection rays (every launch)
  unsigned long long light_entries;          // light connection samples of committed tiles
  unsigned long long light_vertex_entries;   // light subpath vertices of committed tiles
  unsigned long long shadow_entries;     // shadow rays of committed tiles
  unsigned long long shadow_traced;      // listed (traced) shadow rays of committed tiles
  unsigned long long wave_total[MAXD + 2];  // rays per depth wave of committed tiles
  // traversal work of the closest-hit (0) and shadow (1) kernels: node visits,
  // quad, sphere and triangle tests (every launch, committed or not)
  unsigned long long trace_work[2][4];
  unsigned int overflow;       // this tile overflowed the arena
  unsigned int any_overflow;   // some tile of this iteration overflowed
  unsigned long long demand;   // rays the tile needed (may exceed the arena)
  unsigned long long rays, vertices, est_vertices;
  unsigned long long entries;  // arena slots processed by committed tiles (all waves)
  double sum_beta[NT];
  // image statistics: per slot, the sums over pixels of the running mean's
  // channels (0..2) and of the pixels' squared relative errors (3)
  double img_part[IMG_SLOTS][4];
  float img_part32[IMG_SLOTS][4];  // the same sums in float32 (float32 statistics)
  double vi_sum;                   // the V_I sum: the slots' total less the rejected pixels' terms
  float vi_sum32;
  double VI, CI;               // results of the last image-stats pass
  int vi_dropped;              // pixels left out of the V_I mean
  unsigned int check_flags;    // MARS_CHECK_* bits of failed index checks (checked builds)
};

// technique t's slot is in use: slot 2 holds the guided technique or the light
// connection (they exclude each other)
__host__ __device__ __forceinline__ bool slot_on(int techniques, int t) {
  return t == 2 ? (techniques & (MARS_TECH_GUIDED | MARS_TECH_LIGHT)) != 0 : ((techniques >> t) & 1) != 0;
}

// Index checks of the checked build (-DMARS_CHECKED, libmars_checked.so): an
// index a kernel computed is tested against the buffer it addresses; a failed
// test sets its MARS_CHECK_* bit in the counters and the caller skips the
// access.  Regular builds compile every check to `true`.
__device__ __forceinline__ bool chk(bool ok, unsigned int bit, DevCounters* ctr) {
#ifdef MARS_CHECKED
  if (!ok) atomicOr(&ctr->check_flags, bit);
  return ok;
#else
  (void)bit;
  (void)ctr;
  return true;
#endif
}

struct DevCache {
  int grid_n, n_cells, techniques, max_depth, bits;
  int n_pixels;
  float4* cnt;          // [cells][3][2]: (q_rr xyz, valid), (q_s xyz, 0)
  double* stats;        // [8][cells][3] (float64 statistics, structure of arrays)
  float* stats32;       // [cells][3][8] (float32 statistics; then stats is null)
  float* guide_hist;    // [cells][256]
  float* guide_cdf;     // [cells][256]
  uint8_t* guide_dirty; // [cells] 1: deposits since the last CDF rebuild
  float4* est;          // [pixels] pixel estimate
  float4* run_sum;      // [pixels]
  float4* img;          // [pixels] this iteration's image
  DevCounters* ctr;
  unsigned int* tile_status;  // [max tiles] overflow per tile of the current attempt
  // adaptive octree over the scene box (oct_nodes null: the uniform grid).
  // node >= 0: first of its 8 children (octant x | y << 1 | z << 2); < 0: leaf ~cell
  int* oct_nodes;       // [oct_cap_nodes]
  int* oct_leaf_level;  // [n_cells]
  int* oct_leaf_node;   // [n_cells] node holding the leaf
  int* oct_meta;        // [0] nodes, [1] leaves, [2] splits of the last refinement
  int* oct_split;       // [n_cells / 7 + 1] parent cell of split s
  float* oct_leaf_n;    // [n_cells] samples of the last iteration per leaf
  int oct_cap_nodes;
  float split_samples;
  float4* comb;                 // [pixels] inverse-variance weighted image sum
  double* comb_w;               // its weight sum
  // [3] sums of V_I and C_I over the iterations whose image statistics ran since
  // the last update, and their count: the update takes the means
  double* img_acc;
  unsigned long long* topk;     // [IMG_TOPK_BLOCKS * MAX_DROP] brightness candidates
};
constexpr int MAX_DROP = MARS_MAX_DROP_BRIGHTEST;
constexpr int IMG_TOPK_BLOCKS = 1024;
constexpr int OCT_LMAX = MARS_OCTREE_MAX_LEVEL;

// Arguments of one tile of one iteration.  They live in device memory (one
// slot per tile) and every kernel reads them from there, so that a recorded
// iteration graph is replayed with the next iteration's values.
struct IterArgs {
  uint32_t seed, job, iteration;
  int mode, aware, collect, has_estimate;
  float clamp_lo, clamp_hi, outlier;
  float max_mult;  // path multiplicity cap (0: none)
  int tile_begin, tile_end, tile_slot;
  int n_prev;      // iterations already summed into the running image
  int drop_k;      // V_I leaves out the drop_k brightest pixels (0: outlier clamp)
  int combine;     // 0 none, 1 add to, 2 restart the inverse-variance combination
};

// Launch shape of the four per-wave kernels: threads per block (a multiple of
// 32, at most 256) and grid size in blocks, the same for every depth wave (a
// persistent grid; sizing each wave's grid from the previous iteration's wave
// sizes measured no faster for small waves and starved the growing waves of
// the first MARS iterations).  Every kernel strides over its wave in chunks
// of 32 slots, so results do not depend on the shape.
// (the light connection kernel runs with the shadow kernel's shape)
enum { WK_TRACE = 0, WK_SHADE = 1, WK_SHADOW = 2, WK_REVERSE = 3, WAVE_KERNELS = 4 };
struct WaveLaunch {
  int threads[WAVE_KERNELS];
  int variant[WAVE_KERNELS];               // register-cap variant (wave_variant_registers)
  int grid[WAVE_KERNELS];                  // persistent grid: SMs x resident blocks
};

// the light connection kernel of wave d (bdpt.cu)
cudaError_t launch_light(const DevScene& s, const DevCache& c, const Arena& a, const IterArgs* it, int variant,
                         int grid, int threads, int d, cudaStream_t st);
int light_variants();

// launch wrappers (render.cu)
// it: device pointer to the tile's arguments
// side2: the light connection kernels' stream (light connections only; null:
// they run on side); sync: D + 2 events
cudaError_t launch_tile(const DevScene& s, const DevCache& c, const Arena& a, const IterArgs* it,
                        const WaveLaunch& L, cudaStream_t st, cudaStream_t side, cudaStream_t side2,
                        const cudaEvent_t* sync, cudaEvent_t* ev);
// adds a second tile lane's iteration totals into the first lane's counters
cudaError_t launch_merge_lanes(DevCounters* dst, DevCounters* src, cudaStream_t st);
// resident blocks per SM of each wave kernel at the given block sizes and variants
cudaError_t wave_occupancy(const int threads[WAVE_KERNELS], const int variant[WAVE_KERNELS],
                           int blocks_per_sm[WAVE_KERNELS]);
int wave_variants(int kernel);                    // compiled register-cap variants of a wave kernel
int wave_variant_registers(int kernel, int v);    // its register cap (0: the compiler's choice)
bool wave_threads_ok(int threads);
int tile_launches(int max_depth, int techniques);  // kernels launch_tile issues
// image statistics (stats.cu)
// it: device pointer to the iteration's arguments (n_prev, outlier, drop_k,
// combine); drop / combine: whether the brightest-pixel rejection and the
// progressive combination kernels run
cudaError_t launch_image_stats(const DevCache& c, int width, int height, const IterArgs* it,
                               float* image_out_dev, bool drop, bool combine, int num_sms, cudaStream_t st);
// the combined image divided by its weight sum, packed rgb, into out (device)
cudaError_t launch_combined_out(const DevCache& c, int npix, float* out, cudaStream_t st);
cudaError_t launch_image_copy(const DevCache& c, int npix, float* out, cudaStream_t st);
// the iteration image of pixels [p0, p1) only, packed rgb, into out (device; the whole frame's layout)
cudaError_t launch_image_copy_range(const DevCache& c, int p0, int p1, float* out, cudaStream_t st);
cudaError_t launch_update(const DevCache& c, int num_sms, cudaStream_t st);
// octree refinement after an update (stats.cu): leaf_samples must run before
// launch_update (which zeroes the statistics), refine after it
cudaError_t launch_leaf_samples(const DevCache& c, cudaStream_t st);
cudaError_t launch_octree_refine(const DevCache& c, int num_sms, cudaStream_t st);
// scene build (scene.cu)
// SAH build on the host from the primitive boxes (2 float4 per primitive):
// n - 1 internal nodes, root 0; false if n < 2 (scene.cu)
bool build_bvh_sah(const std::vector<float4>& boxes, int n, std::vector<BvhNode>& nodes);
cudaError_t build_bvh(const float4* d_prims, int n, const float lo[3], const float ext[3], BvhNode* d_nodes,
                      cudaStream_t st, std::string* err);

}  // namespace mars
