// abi_internal.h -- host-side object layouts behind the opaque ABI handles.
#pragma once

#include <cuda_runtime.h>

#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace mars {

// Owned deep copy of a mars_scene_desc (the server keeps one per job).
struct SceneDescCopy {
  std::vector<double> quads, spheres, tris, materials;
  std::vector<int32_t> quad_mat, sphere_mat, tri_mat;
  mars_scene_desc desc{};
  void assign(const mars_scene_desc* d) {
    quads.assign(d->quads, d->quads + 9 * (size_t)d->n_quads);
    spheres.assign(d->spheres, d->spheres + 4 * (size_t)d->n_spheres);
    tris.assign(d->tris, d->tris + 9 * (size_t)d->n_tris);
    materials.assign(d->materials, d->materials + 8 * (size_t)d->n_materials);
    quad_mat.assign(d->quad_mat, d->quad_mat + d->n_quads);
    sphere_mat.assign(d->sphere_mat, d->sphere_mat + d->n_spheres);
    tri_mat.assign(d->tri_mat, d->tri_mat + d->n_tris);
    desc = *d;
    desc.quads = quads.data();
    desc.spheres = spheres.data();
    desc.tris = tris.data();
    desc.materials = materials.data();
    desc.quad_mat = quad_mat.data();
    desc.sphere_mat = sphere_mat.data();
    desc.tri_mat = tri_mat.data();
  }
};

mars_status set_error(mars_status s, const char* fmt, ...);

// An NVTX range over a scope: the library's stages show up by name in
// profilers (ncu --nvtx filters kernels by them); without a tool attached the
// calls do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// What a recorded iteration graph depends on besides the per-tile arguments,
// which the kernels read from device memory: it is replayed while these are
// unchanged and recorded again otherwise.
struct GraphKey {
  bool update_estimate = false, drop = false, combine = false;
  int tiles = 0;
  float* dev_out = nullptr;
  int64_t r0 = 0, r1 = 0;  // pixel range (the image copy of a range is recorded with its bounds)
  WaveLaunch L{};
  bool operator==(const GraphKey& o) const {
    return update_estimate == o.update_estimate && drop == o.drop && combine == o.combine && tiles == o.tiles &&
           dev_out == o.dev_out && r0 == o.r0 && r1 == o.r1 && std::memcmp(&L, &o.L, sizeof(WaveLaunch)) == 0;
  }
};

// Device memory of scenes and caches comes from the device's stream-ordered
// memory pool (cudaMallocAsync / cudaFreeAsync), which keeps released memory
// for reuse: creating and destroying objects while other streams render
// neither maps nor unmaps memory nor synchronises the device.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);
// Page-locked host buffers for the per-iteration status copies, kept in a
// process-wide free list (cudaMallocHost / cudaFreeHost are slow and serialise).
void* pinned_acquire(size_t bytes);
void pinned_release(void* p, size_t bytes);

}  // namespace mars

struct mars_scene {
  int device = 0;
  int num_sms = 0;
  int width = 0, height = 0, n_prims = 0, n_lights = 0;
  mars::DevScene ds{};
  float4* d_prims = nullptr;
  float4* d_boxes = nullptr;
  mars::BvhNode* d_nodes = nullptr;
  mars::Bvh4Node* d_nodes4 = nullptr;
  float4* d_mats = nullptr;
  float4* d_lights = nullptr;
  uint64_t device_bytes = 0;
  mars::SceneDescCopy desc_copy;
  cudaStream_t stream = nullptr;  // the stream it was created on (released there)
};

struct mars_cache {
  const mars_scene* scene = nullptr;
  int device = 0;
  int grid_n = 0, techniques = 0, max_depth = 0;
  int64_t cells = 0, pixels = 0;
  mars::Arena arena{};
  mars::DevCache dc{};
  float4* d_cnt = nullptr;
  double* d_stats = nullptr;
  float* d_stats32 = nullptr;  // float32 statistics variant (then d_stats is null)
  bool fp32_stats = false;
  float* d_hist = nullptr;
  float* d_cdf = nullptr;
  uint8_t* d_guide_dirty = nullptr;
  int* d_oct_nodes = nullptr;   // adaptive octree (MARS_CACHE_OCTREE)
  int* d_oct_level = nullptr;
  int* d_oct_lnode = nullptr;
  int* d_oct_meta = nullptr;
  int* d_oct_split = nullptr;
  float* d_oct_leaf_n = nullptr;
  int oct_cap_nodes = 0;
  float4* d_est = nullptr;
  float4* d_run = nullptr;
  float4* d_img = nullptr;
  mars::DevCounters* d_ctr = nullptr;
  unsigned int* d_tile_status = nullptr;
  mars::DevCounters* h_ctr = nullptr;
  unsigned int* h_tile_status = nullptr;
  int max_tiles = 0;
  int next_tiles = 1;
  int n_iterations = 0;
  bool has_estimate = false;
  bool poisoned = false;
  uint64_t device_bytes = 0;
  std::vector<cudaEvent_t> events;  // profiling events, grown on demand
  cudaStream_t last_stream = nullptr;  // the stream of the last call that used the cache
  cudaStream_t side = nullptr;         // second stream: NEE shadow rays overlap the next waves
  cudaStream_t side2 = nullptr;        // third stream: light connection kernels (light connections only)
  std::vector<cudaEvent_t> sync_events;  // D + 2 cross-stream events (no timing)
  mars::WaveLaunch launch{};        // launch shape of the per-wave kernels
  int blocks_per_sm[mars::WAVE_KERNELS] = {0, 0, 0, 0};  // 0: occupancy maximum
  uint64_t last_entries = 0;  // arena slots the last iteration used (tile planning)
  double last_need = 0.0;     // ... as a fraction of the arena (the larger of rays and shadow rays)
  // Tile lanes: the pixel tiles of an iteration are dealt round-robin to
  // `lanes` lanes; lane l renders on its own streams with its own counters
  // (d_ctr[l]) in its own 1/lanes share of the arena, so the two lanes' wave
  // kernels fill each other's idle SMs (the small deep waves leave most of the
  // GPU idle); lane 1's totals are merged into lane 0's before the image pass.
  static constexpr int kMaxLanes = 4;
  int lanes = 1;                    // lanes with streams and counters (as created)
  int use_lanes = 1;                // lanes an iteration may use (<= lanes)
  int64_t lane_min_pixels = 1 << 17;  // smallest image split over the lanes
  // lanes 1..lanes-1: rendering stream, shadow stream, D + 1 fork / join
  // events between them, and the event that joins the lane to the caller's
  // stream; fork_ev forks all of them from it
  std::vector<cudaStream_t> lane_st, lane_side, lane_side2;
  std::vector<std::vector<cudaEvent_t>> lane_sync;
  std::vector<cudaEvent_t> join_ev;
  cudaEvent_t fork_ev = nullptr;
  // per-tile iteration arguments: written to the pinned slots, copied to the
  // device slots before the launches, read there by every kernel
  mars::IterArgs* h_args = nullptr;
  mars::IterArgs* d_args = nullptr;
  float* d_host_stage = nullptr;  // packed rgb image for image_on_host (first use)
  float4* d_comb = nullptr;       // inverse-variance weighted image sum
  double* d_comb_w = nullptr;     // its weight sum
  double* d_img_acc = nullptr;    // V_I and C_I sums since the last update, and their count
  unsigned long long* d_topk = nullptr;  // brightest-pixel candidates
  // the recorded single-tile iteration graph (MARS_CACHE_NO_GRAPHS: none)
  bool use_graphs = true;
  cudaGraphExec_t graph_exec = nullptr;
  mars::GraphKey graph_key{};
  int graph_captures = 0;
};

namespace mars {
mars_status scene_create_impl(const mars_scene_desc* d, cudaStream_t st, mars_scene** out);
void scene_destroy_impl(mars_scene* s);
mars_status cache_create_impl(const mars_scene* s, const mars_cache_desc* d, cudaStream_t st, mars_cache** out);
void cache_destroy_impl(mars_cache* c);
mars_status render_iteration_impl(mars_cache* c, const mars_iter_params* p, float* image, mars_iter_stats* out,
                                  cudaStream_t st);
mars_status update_counts_impl(mars_cache* c, cudaStream_t st);
mars_status get_state_impl(mars_cache* c, mars_cache_state* s, cudaStream_t st);
uint64_t cache_footprint(int64_t cells, int64_t pixels, int max_depth, int techniques, uint64_t cap);
uint64_t default_capacity(int64_t pixels, int max_depth);
mars_status apply_launch(mars_cache* c, const int threads[WAVE_KERNELS], const int blocks_per_sm[WAVE_KERNELS],
                         const int variant[WAVE_KERNELS]);
}  // namespace mars
