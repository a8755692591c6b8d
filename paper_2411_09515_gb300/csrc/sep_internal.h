// Internal declarations of libsep (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "nvtx3/nvToolsExt.h"
#include "sep.h"

// ---- packed CSR entry ---------------------------------------------------
// One 32-bit word per nonzero of the integration matrix:
//   bits  0..24  pixel index (column of the matrix), < 2^25 (0 for padding)
//   bits 25..26  k - 1 where k / split^2 is the coefficient c_{i,r} (k = 1..4)
//   bit  27      the entry's bin is the pixel's centre bin (threshold bin)
//   bit  28      zero coefficient: the entry exists only to carry bit 27
//   bit  29      padding (no pixel): per-tile runs are padded to 8 entries
namespace sep {
// Restores the calling thread's current device when a C-ABI entry point
// returns: entry points select their context's device for their own calls
// and leave the caller's selection as they found it.
struct DeviceGuard {
  int dev = -1;
  DeviceGuard() {
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (dev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != dev) cudaSetDevice(dev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// An NVTX range named after the C-ABI entry point for the duration of the
// call (a profiler shows each library call on the host timeline; without a
// tool attached a push and a pop cost a few nanoseconds).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr uint32_t kColBits = 25;
constexpr uint32_t kColMask = (1u << kColBits) - 1u;
constexpr uint32_t kKShift = 25;
constexpr uint32_t kCentre = 1u << 27;
constexpr uint32_t kZero = 1u << 28;
constexpr uint32_t kPad = 1u << 29;

// Host-built matrix (own FP64 implementation of Section 2.2's coefficients).
struct HostCsr {
  int32_t rows = 0, cols = 0, nbins = 0, split = 1;
  double lo = 0, hi = 0;
  std::vector<int32_t> rowptr;   // [nbins + 1], multiples of 8
  std::vector<int32_t> grp;      // [nbins][4]: end of coefficient class 0..3 within the row
  std::vector<uint32_t> ent;     // [nnz] packed
  std::vector<float> coef;       // [nnz] c_{i,r} (0 for centre-only entries)
  std::vector<int32_t> cpix;     // [nnz] pixel of a centre entry (it carries its pixel's centre bin), else -1
  std::vector<int32_t> interp_a; // [npix] lower bin of the pixel centre's interpolation (densification)
  std::vector<float> interp_t;   // [npix] its weight on the upper bin, in [0, 1)
  std::vector<float> w;          // [nnz] c * norm (only with a norm)
  std::vector<int32_t> bop;      // [npix] centre bin, -1 masked
  std::vector<float> centers;    // [nbins]
  int32_t max_row = 0;
  // staging order of the pixels (the order of the entries inside each
  // coefficient group of a row)
  int64_t npos = 0;                 // pixels with an entry
  int32_t tiles_x = 0, tiles_y = 0;
  std::vector<int32_t> perm_inv;    // [npos] pixel of each staging position
  std::vector<int32_t> pos_of;      // [npix] staging position of each pixel, -1 if none
  std::vector<int16_t> tile_rank;   // [npix] position inside its tile, -1 if none
  std::vector<int32_t> tile_base;   // [tiles + 1] first position of each tile
  // staged copy of a frame (one value per entry, slot = entry index)
  std::vector<int32_t> slot_of;     // [npix] slot of the pixel's centre entry, -1 if none
  std::vector<int32_t> tile_ebase;  // [tiles + 1] first scatter pair of each tile
  std::vector<int32_t> tile_sc;     // [nnz][2] (slot, pixel index in the tile or -1: padding), by tile
};

constexpr int kTileH = 64, kTileW = 64;   // staging tiles (rows x columns)

// Returns an empty string on success, else the reason.
std::string build_csr_host(const sep_geometry& g, const uint8_t* mask, const float* norm, HostCsr* out);
// Checks of a matrix in the export layout (sep_csr_validate) and of the
// packed layout the kernels read; empty on success, else the first violation.
std::string validate_matrix(const int32_t* rowptr, const int32_t* col, const float* coef, const int32_t* bop,
                            int32_t nbins, int64_t nnz, int64_t npix);
std::string validate_host_csr(const HostCsr& h);

// ---- kernel launch parameters -------------------------------------------
struct ClipArgs {
  const int32_t* bin_list; // bins handled by this launch (blockIdx.x indexes it); null = all, in order
  const int32_t* rowptr;
  const int32_t* grp;      // [nbins][4] class ends within a row
  const uint32_t* ent;     // packed entries: staging position + flags
  const float* w;          // per-entry weight c * norm (NORM variant)
  const float* stage;      // staged values [n_frames][npos] (npos here: the row stride)
  int64_t npos;
  int32_t nbins, n_frames, frames_per_cta, cap;
  int32_t n_iter;
  float k_clip, k_pick;
  int32_t cutoff = 0;      // SEP_CUTOFF_*: fixed k_clip, or Eq. 20 for each set's size
  int32_t error_model = 0; // SEP_ERROR_*: azimuthal, Poisson or hybrid deviation
  float dark_var = 0.0f;   // dark variance of the Poisson model (Eq. 3)
  float* mean;
  float* sigma;
  int32_t* count;
  float* bounds;           // optional [F][B][2]
  int32_t* iters;          // optional [F][B]
  float* thr_out;          // optional [F][B] sparsification thresholds (Section 3)
  // optional kept-pixel marking (Section 3) at the end of each bin's clip:
  // cpix[e] = pixel of entry e if the entry carries its pixel's centre bin,
  // else -1; a centre entry whose value exceeds the bin's threshold sets its
  // pixel's bit in row f of bitmap (words per frame). Null bitmap = no marking.
  const int32_t* cpix = nullptr;
  uint32_t* bitmap = nullptr;
  int64_t words = 0;
  // mixed batches: per launch frame, the first output row (in bins) of its
  // profile; null = rows f * nbins
  const int64_t* orow = nullptr;
  // surrogate: record features + targets (training data), or place the
  // first core from the prediction
  float* rec_feat = nullptr;           // [rows][20]
  float* rec_target = nullptr;         // [rows][2]
  const __nv_bfloat16* mlp_w = nullptr;
  const float* mlp_norm = nullptr;
  unsigned long long* surr_stats = nullptr;   // [2]: bins whose predicted core held, bins that re-placed it
  int32_t tcap = 0;                    // tail slots per thread of the tail-replay kernel (set at launch)
  // persistent launch: each CTA takes units (a bin of the launch and a group
  // of frames_per_cta frames) from the counter *queue, which the launch
  // zeroes, until none is left; null: one unit per CTA
  int32_t* queue = nullptr;
  int32_t units_x = 0, units = 0;      // bins of the launch, units in all (set at launch)
  unsigned long long* clip_stats = nullptr;   // [SEP_CLIP_STATS] counters of the tail replay, or null
};

struct StageArgs {         // correction + staging of a batch (k_stage)
  const void* frames;      // contiguous [n_frames][npix], or
  const uint64_t* fptr;    // per frame address (mixed batches), may be null
  int64_t npix, npos;      // npos: the staged row stride (slots, >= nnz)
  int32_t rows, cols, tiles_x, tiles_y;
  int32_t n_frames, frames_per_cta;
  const float* ped;        // [3][npix] (raw input)
  const float* gain;       // [3][npix]
  const float* norm;       // [npix] or null
  const int32_t* tile_ebase;   // [tiles + 1]
  const int2* tile_sc;         // [nnz] (slot, pixel index in the tile or -1 for padding)
  float* stage;            // [n_frames][npos]: value of entry e at slot e
};

struct PixArgs {           // what the consumers need to recompute a pixel value
  const void* frames;
  int64_t npix;
  int32_t rows, cols, dtype;
  const float* ped;
  const float* gain;
  const float* norm;       // may be null
  const int32_t* bop;      // [npix], -1 masked
  // mixed batches: per launch frame, its address, its index among the
  // call's frames (rows of the kept / peak outputs) and its profile row
  const uint64_t* fptr = nullptr;
  const int32_t* fidx = nullptr;
  const int64_t* orow = nullptr;
  // staged values of the batch ([frame][npos], frame = launch index), when
  // the call staged them: read instead of recomputing from the raw word
  const float* stage = nullptr;
  const int32_t* pos_of = nullptr;   // [npix] staging position, -1 if not staged
  int64_t npos = 0;
  // background at the pixel centre interpolated between bin centres (lower
  // bin, weight on the upper bin, per pixel); null: the centre bin's level
  const int32_t* ia = nullptr;
  const float* it = nullptr;
};

// mode 0: set the kernel's shared-memory attribute and launch; 1: attribute
// only (call before a stream capture); 2: launch only.
cudaError_t launch_integrate_clip(const ClipArgs& a, int n_ctas, int tpb, bool split, bool has_norm,
                                  int32_t precision, int mode, cudaStream_t s);
cudaError_t launch_stage(const StageArgs& a, int32_t dtype, bool has_norm, cudaStream_t s);
size_t clip_smem_bytes(int32_t cap, bool weighted);
// Tail slots per thread the tail-replay clip kernel asks for (rows of `cap`
// entries, `tpb` threads); fewer are used where shared memory runs out.
int32_t clip_tail_slots(int32_t cap, int32_t tpb);
constexpr int kClipStaticSmem = 2048;   // static shared memory of the clip kernels (upper bound)
cudaError_t launch_thresholds(const float* mean, const float* sigma, float k_pick, int64_t n, float* thr,
                              cudaStream_t s);
// Kept-pixel bitmap with each pixel's threshold taken from the profile
// interpolated at its centre (p.ia, p.it); every word of the n_frames rows
// is written. Profile rows: p.orow[f] when set, else f * nbins.
cudaError_t launch_mark_interp(const PixArgs& p, int32_t n_frames, int32_t nbins, const float* mean,
                               const float* sigma, float k_pick, uint32_t* bitmap, int64_t words, cudaStream_t s);
// Dense frames from their sparse form (Section 3): background by bin, then
// the kept pixels' values.
cudaError_t launch_densify(const int32_t* bop, int64_t npix, int32_t nbins, int32_t n_frames, const float* mean,
                           const float* sigma, const int32_t* idx, const float* val, int64_t cap,
                           const int32_t* n_kept, const float* noise, float fill, const int32_t* interp_a,
                           const float* interp_t, float* out, cudaStream_t s);
// Veto (Section 4): ascending list of the frames with >= min_peaks peaks.
cudaError_t launch_veto(int32_t n_frames, const int32_t* n_peaks, int32_t min_peaks, int32_t* list, int32_t* n_pass,
                        cudaStream_t s);
// Rows list[j] of src to rows j of dst, j < *n_pass (row_bytes a multiple of 4).
cudaError_t launch_compact_rows(int32_t n_frames, const int32_t* list, const int32_t* n_pass, int64_t row_bytes,
                                const void* src, void* dst, cudaStream_t s);
// Staged values back to image order (NaN where a pixel has no position).
cudaError_t launch_unstage(const float* stage, int64_t stride, const int32_t* pos_of, int64_t npix, int32_t n_frames,
                           float* out, cudaStream_t s);
cudaError_t launch_mark(const PixArgs& p, int32_t n_frames, int32_t nbins, const float* thr, uint32_t* bitmap,
                        int64_t words, cudaStream_t s);
// Ordered compaction of the kept-pixel bitmap (two launches; scratch holds
// per-tile counts) and peak picking over the kept list (two launches;
// scratch holds flag bits and per-chunk counts). consumer_scratch_words gives
// the int32 scratch both need.
cudaError_t launch_compact(const PixArgs& p, int32_t n_frames, const uint32_t* bitmap, int64_t words,
                           int32_t* idx, float* val, int64_t cap, int32_t* n_kept, int32_t* scratch,
                           int32_t* status, cudaStream_t s);
int64_t consumer_scratch_words(int32_t n_frames, int64_t words, int64_t kcap);
cudaError_t launch_scatter_list(int32_t n_frames, const int32_t* idx, const int32_t* n_kept, int64_t kcap,
                                int64_t npix, uint32_t* bitmap, int64_t words, cudaStream_t s);
cudaError_t launch_peaks(const PixArgs& p, int32_t n_frames, int32_t nbins, const float* mean, const float* sigma,
                         const uint32_t* bitmap, int64_t words, const int32_t* idx,
                         const int32_t* n_kept, int64_t kcap, int32_t patch, int32_t min_count,
                         sep_peak* peaks, int64_t pcap, int32_t* n_peaks, int32_t* scratch, int32_t* status,
                         cudaStream_t s);
// The argument and parameter checks every batch entry point runs (context,
// matrix, calibration, frames, dtype, frame count, sep_params); on success
// the context's device is current.
sep_status check_call(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames, int32_t dtype,
                      int32_t n_frames, const sep_params* params);

}  // namespace sep

// ---- handles --------------------------------------------------------------
struct sep_graph_entry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

struct sep_ctx {
  int32_t device = 0;
  int num_sms = 0;
  // fork/join of the clip launches of several size classes
  cudaStream_t aux[4] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[4] = {};
  int32_t* d_status = nullptr;
  std::string err;
  // scratch owned by the context, grown on demand (never inside a capture)
  uint32_t* d_bitmap = nullptr;
  size_t bitmap_words = 0;
  float* d_thr = nullptr;
  size_t thr_len = 0;
  int32_t* d_aux = nullptr;    // consumer scratch (tile counts, flag bits)
  size_t aux_len = 0;
  int64_t* d_desc = nullptr;   // mixed batches: per-frame descriptor table
  int64_t* h_desc = nullptr;   // its pinned staging copy
  size_t desc_len = 0;
  unsigned long long* d_surr = nullptr;   // surrogate counters: settled, fell back
  unsigned long long* d_clip_stats = nullptr;   // [SEP_CLIP_STATS] tail-replay counters
  // work-queue counters of the persistent clip launches, taken in turn (one
  // per launch in flight: a call forks at most 4 x 4 clip launches)
  static constexpr int kQueueSlots = 64;
  int32_t* d_queue = nullptr;
  uint32_t queue_next = 0;
  bool clip_stats_on = false;                   // clip launches count into d_clip_stats
  float* d_stage = nullptr;    // staged pixel values of the batch in flight
  size_t stage_len = 0;
  // host pipeline (sep_process_host): chunk slots of frames + outputs
  unsigned char* d_pipe = nullptr;
  size_t pipe_len = 0;
  static constexpr int kCopyStreams = 1;   // streams a chunk's copy-in is split over (more measured slower)
  static constexpr int kSlots = 3;         // chunks in flight: copy-in, compute, copy-out
  cudaStream_t s_in[kCopyStreams] = {}, s_out = nullptr;
  cudaEvent_t ev_in[kSlots][kCopyStreams] = {}, ev_done[kSlots] = {}, ev_out[kSlots] = {}, ev_start = nullptr;
  // captured batches, keyed by every launch argument
  std::map<std::vector<uint64_t>, sep_graph_entry> graphs;
  uint64_t use_clock = 0;
};

// One size class of bins for the clip kernel: its own block size and
// shared-memory capacity (the largest row in the class), big rows first.
struct sep_clip_class {
  int32_t* d_bins = nullptr;
  int32_t n_bins = 0;
  int32_t cap = 0;
  int32_t tpb = 256;
  int32_t threshold = 0;   // rows with more entries than the previous class's threshold, up to this
};

struct sep_csr {
  sep_ctx* ctx = nullptr;
  sep::HostCsr h;
  std::vector<sep_clip_class> plan;   // empty = one class of every bin at 256 threads
  uint64_t plan_version = 0;
  int64_t npix = 0, nnz = 0;
  bool has_norm = false;   // values are divided by a norm (Eq. 1)
  bool weighted = false;   // per-entry weights c * norm (a norm, or exact area fractions)
  int32_t* d_rowptr = nullptr;
  uint32_t* d_ent = nullptr;
  int32_t* d_cpix = nullptr;          // pixel of each centre entry, else -1
  int32_t* d_interp_a = nullptr;      // radial interpolation of the background (densification)
  float* d_interp_t = nullptr;
  float* d_w = nullptr;
  float* d_norm = nullptr;
  int32_t* d_bop = nullptr;
  int32_t* d_grp = nullptr;
  int32_t* d_pos_of = nullptr;        // slot of each pixel's centre entry in a staged row, -1 if none
  int32_t* d_tile_ebase = nullptr;
  int2* d_tile_sc = nullptr;
  const sep_model* model = nullptr;   // surrogate attached by sep_csr_attach_model
};

struct sep_model {
  sep_ctx* ctx = nullptr;
  float* d_params = nullptr;      // FP32 master parameters
  __nv_bfloat16* d_wbf = nullptr; // BF16 copy read by every forward / backward
  __nv_bfloat16* d_wbt = nullptr; // the same, W1 and W2 input-major (the clip kernel's inference)
  float* d_m = nullptr;           // Adam moments
  float* d_v = nullptr;
  float* d_grad = nullptr;
  float* d_loss = nullptr;
  float* d_norm = nullptr;        // feature / target normalisation (device copy)
  float norm[SEP_MLP_NORM] = {};
  int64_t step = 0;
};

struct sep_calib {
  sep_ctx* ctx = nullptr;
  const sep_csr* csr = nullptr;
  int64_t npix = 0;
  float* d_ped = nullptr;
  float* d_gain = nullptr;
};
