// dkm_host.h -- internal declarations shared by the libdkm translation units:
// the kernel launchers (defined next to their kernels) and the context.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/dkm.h"
#include "dkm_device.cuh"

namespace dkm {

// dkm_setup.cu
cudaError_t launch_bbox(const float* p, int d, const int64_t* seg, int B, int64_t max_rows,
                        CloudRun* crun, DevState* st, int which, int d_ctx, cudaStream_t s);
cudaError_t launch_exponents(const Cloud* clouds, CloudRun* crun, int B, cudaStream_t s);
cudaError_t launch_morton(const float* p, int64_t n, int d, const int64_t* seg, int B,
                          const Cloud* clouds, int mb, uint32_t* keys, int bits_lo, int bits_hi,
                          void* scratch, cudaStream_t s);
size_t rs_scratch_bytes(int64_t n);
cudaError_t launch_radix_sort(uint32_t* keys[2], uint32_t* vals[2], int64_t n, int bits_lo,
                              int bits_hi, void* scratch, DevState* st, int* final_buf,
                              cudaStream_t s);
cudaError_t launch_sort_wait_selftest(uint32_t* keys[2], uint32_t* vals[2], int64_t n,
                                      void* scratch, DevState* st, cudaStream_t s);
cudaError_t launch_gather(const float* p, int64_t n, int d, const uint32_t* order, float* xs,
                          float* ys, float* zs, int64_t n_pad, cudaStream_t s);
cudaError_t launch_levels(const uint32_t* keys, int64_t n, int d, int mb, int B,
                          unsigned long long* hist, cudaStream_t s);
cudaError_t launch_lattice(Cloud* clouds, const CloudRun* crun, int B, int d, int mb,
                           cudaStream_t s);
size_t tiles_scratch_words(int n_windows);
cudaError_t launch_tiles(const uint32_t* keys, int64_t n, Cloud* clouds, int d, int mb, int B,
                         int cut_div, const unsigned long long* level_hist, int n_windows,
                         const float* xs, const float* ys, const float* zs, unsigned* scratch,
                         int tiles_cap, int2* tiles, float4* tbox, int* tcloud, int* tfirst,
                         int* n_tiles, cudaStream_t s);

// dkm_iter.cu
cudaError_t launch_reset_run(const IterArgs& A, cudaStream_t s);
cudaError_t launch_centroids(const IterArgs& A, int mode, int t, int d, const float* user_c,
                             int insert, int par, int32_t* counts_out, cudaStream_t s);
cudaError_t launch_search(const IterArgs& A, int par, int d, cudaStream_t s);
cudaError_t launch_seed_refs(const IterArgs& A, int par, int d, cudaStream_t s);
cudaError_t launch_assign(const IterArgs& A, int d, int brute, cudaStream_t s);
cudaError_t launch_collect(const IterArgs& A, int t, cudaStream_t s);
cudaError_t launch_accum_labels(const IterArgs& A, int d, const int32_t* ulab,
                                const uint32_t* perm, cudaStream_t s);
cudaError_t launch_finalize(const IterArgs& A, int d, const uint32_t* perm, int32_t* labels_out,
                            int do_sse, cudaStream_t s);
cudaError_t launch_export(const float4* cw, int k, int d, float* out, cudaStream_t s);
cudaError_t launch_cbound(const IterArgs& A, int par, int d, int use_ub, cudaStream_t s);
cudaError_t launch_unit_boxes(const float4* tbox, const int* tcloud, const int* ufirst,
                              int n_units, float4* ubox, int* ucloud, int* tunit,
                              cudaStream_t s);

// dkm_api.cu: set the calling thread's dkm_last_error() message
void dkm_set_last_error(const char* msg);

}  // namespace dkm

// A context holds B >= 1 independent k-means problems ("clouds") over one
// concatenated point array; the single-cloud API is the case B = 1.
struct dkm_ctx {
  int64_t n = 0;               // total points
  int d = 0;
  int k = 0;                   // total centroids (sum of ks)
  int B = 1;                   // clouds
  std::vector<int64_t> offsets;   // B + 1 point offsets
  std::vector<int> ks;            // B centroid counts
  std::vector<int64_t> coffs;     // B + 1 centroid offsets
  int64_t max_n_b = 0, max_k_b = 0;
  int mb = 10;                 // Morton bits per axis
  int key_bits = 30;           // significant bits of the sort key
  dkm_options opts{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int n_blocks = 0;            // 2048-point padding blocks
  int n_windows = 0;           // 256-point windows
  int tiles_cap = 0;           // capacity of the tile arrays
  int n_tiles = 0;             // tiles of the current point index
  int tile_level = 0;          // Morton level whose cube boundaries cut cloud 0's tiles
  int cut_div = 2;             // cube cuts may add n_windows / cut_div tiles per cloud
  int unit_g = 1;              // tiles per search unit
  int n_units = 0;             // search units of the current tiling
  float cpc = 1.0f;            // grid cells per centroid (before the budget cap)
  int64_t n_pad = 0;
  int64_t max_cells = 0;       // grid capacity the arena was sized for
  int64_t total_cells = 0;     // cells of the current grids
  dkm_plan_info plan{};
  std::vector<dkm::Cloud> h_clouds;               // host copy of the cloud table
  std::vector<float> h_blo, h_bhi;                // per-cloud point boxes (3 floats each)
  int row_filter_min = 48;     // per-row candidate filtering threshold
  int sort_max = 0;            // sorted early-exit evaluation for lists up to this length
  int stay = 0;                // the bound layer's stay test (tile_group 1 only)
  bool ready = false;          // the point index is valid
  bool lists_seeded = false;   // the candidate-list counters were cleared once
  bool acc_valid = false;      // acc holds the sums of the last dkm_assign

  // device arena
  void* arena = nullptr;
  size_t arena_bytes = 0;
  float *xs = nullptr, *ys = nullptr, *zs = nullptr;
  uint32_t* keys[2] = {nullptr, nullptr};
  uint32_t* vals[2] = {nullptr, nullptr};
  uint32_t* skeys = nullptr;   // sorted keys (one of keys[])
  uint32_t* perm = nullptr;    // sorted position -> original index
  void* rs_scratch = nullptr;  // radix sort: digit counts, tickets, look-back words
  float4* tbox = nullptr;
  int2* tiles = nullptr;
  int* tcloud = nullptr;
  int* tfirst = nullptr;       // per cloud: its first tile
  int* kcloud = nullptr;
  float* cb2 = nullptr;        // per centroid: squared gap to its nearest other centroid
  float* drift = nullptr;      // per centroid: distance moved by the last update
  int* tlab = nullptr;         // per tile: single label of its last pass, or -1
  float4* ubox = nullptr;      // per unit box (unit_g > 1)
  int *ucloud = nullptr, *ufirst = nullptr, *tunit = nullptr;
  unsigned* tl_scratch = nullptr;   // tiling: cut masks, window counts, CTA totals
  unsigned long long* level_hist = nullptr;
  int64_t *doff = nullptr, *dcoff = nullptr;
  dkm::Cloud* clouds = nullptr;
  dkm::CloudRun* crun = nullptr;
  dkm::CloudAcc* cacc = nullptr;
  int32_t* lab = nullptr;
  float4* cw = nullptr;
  dkm::Acc* acc = nullptr;
  dkm::Slot* slots = nullptr;
  dkm::DevState* st = nullptr;
  int* gcnt[2] = {nullptr, nullptr};
  float4* gbkt[2] = {nullptr, nullptr};
  float4* ovf[2] = {nullptr, nullptr};
  int* ovf_cnt[2] = {nullptr, nullptr};
  float4* tlist = nullptr;     // per tile kTileCap candidates of the last search
  int* tcnt = nullptr;
  int* tref = nullptr;         // per unit: the last search's bound-defining centroid
  float* cstage = nullptr;     // k x d centroid staging
  float* cstage2 = nullptr;    // k x d centroid output staging
  int32_t* kstage = nullptr;   // k counts staging

  // pinned host staging: DevState, then B CloudRun, then B Cloud
  void* hpin = nullptr;

  // lazily allocated
  double* sse_hist = nullptr;
  unsigned long long* chg_hist = nullptr;
  int hist_cap = 0;
  float* pstage = nullptr;     // n x d, for host point input
  int32_t* lstage = nullptr;   // n, for host label input / output

  // cached iteration graph
  cudaGraphExec_t gexec = nullptr;
  bool one_shot = false;       // dkm_fit: launch the run directly, no graph
  int g_iters = -1, g_algo = -1, g_early = -1, g_profile = -1;
  dkm::IterArgs g_args{};             // the kernel arguments the graph captured
  std::vector<cudaEvent_t> ev;        // per-pass events of the cached graph
  cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_c = nullptr;
  cudaEvent_t ev_s0 = nullptr, ev_s = nullptr;   // around the last dkm_setup
  bool setup_pending = false;                    // ev_s not read out yet

  dkm_timings timings{};
};
