/*
 * sep.h - C ABI of libsep, the GB300 (sm_103a) signal-separation library.
 *
 * The library implements the per-frame path of Kieffer et al., "Application
 * of signal separation to diffraction image compression and serial
 * crystallography" (arXiv 2411.09515): Jungfrau detector correction,
 * CSR azimuthal integration with per-bin weighted moments, iterative
 * sigma-clipping, sparsification and peak picking.
 *
 * Conventions (every function):
 *  - Frame, output and count buffers passed to compute calls are DEVICE
 *    pointers owned by the caller. Host pointers are only accepted where a
 *    parameter says "_host".
 *  - Handles (sep_ctx, sep_csr, sep_calib) are owned by the library and freed
 *    with the matching *_destroy; destroying NULL is a no-op.
 *  - Compute calls are asynchronous on the given stream (a cudaStream_t;
 *    NULL = the legacy default stream). They return a sep_status for errors
 *    detected on the host before any launch (bad argument, CUDA launch
 *    error). Conditions found on the device (capacity exceeded, a bounded
 *    wait that gave up) are OR-ed into the context's device status word,
 *    read and cleared with sep_get_device_status.
 *  - sep_last_error(ctx) describes the last host-side failure on ctx.
 *  - Calls run on their context's device and leave the calling thread's
 *    current CUDA device as they found it.
 *  - The library never exits, aborts or traps.
 *  - Not thread-safe per context: calls on one sep_ctx must not overlap in
 *    host threads, and their device work must not overlap either (the
 *    context's scratch, staging buffer and work-queue counters serve one
 *    call at a time): issue a context's calls on one stream, or order the
 *    streams with events.
 */
#ifndef SEP_H_
#define SEP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
typedef int32_t sep_status;
#define SEP_OK            0
#define SEP_ERR_ARG       1   /* invalid argument (NULL, size, range, mismatch) */
#define SEP_ERR_CUDA      2   /* a CUDA runtime call or launch failed */
#define SEP_ERR_OOM       3   /* device or host allocation failed */
#define SEP_ERR_CAPACITY  4   /* device flag: more results than the output capacity */
#define SEP_ERR_TIMEOUT   5   /* device flag: a bounded wait gave up */
#define SEP_ERR_CSR       6   /* CSR invalid or a bin too large for the kernels */
#define SEP_ERR_STATE     7   /* handle used with the wrong context/device */

/* device status word bits (sep_get_device_status) */
#define SEP_DEV_CAPACITY  0x1 /* some frame had more kept pixels or peaks than capacity */
#define SEP_DEV_TIMEOUT   0x2

/* ---- enums ------------------------------------------------------------- */
#define SEP_UNIT_2TH_DEG  0   /* scattering angle 2theta, degrees */
#define SEP_UNIT_Q_NM     1   /* q = 4 pi sin(theta) / lambda, nm^-1 */
#define SEP_UNIT_R_MM     2   /* radius on the detector, mm */

#define SEP_DTYPE_F32     0   /* float32 corrected signal (photons) per pixel */
#define SEP_DTYPE_U16_JF  1   /* raw Jungfrau word: 2 gain bits (15:14) + 14-bit ADC */

/* Precision of the per-bin moments (Section 2.2's reductions). One warp
 * owns a bin and frame; each lane sums its share of the row in FP32 about a
 * shift near the mean; the modes differ in how the lanes' sums are merged
 * and the moments finalised:
 * PLAIN:     plain FP32 merges and finalisation.
 * KAHAN:     Kahan-compensated per-lane sums, error-free FP32 pair merges,
 *            double-word (FP32 pair) finalisation.
 * FP64MERGE: FP64 merge across the warp and FP64 finalisation.
 * DWORD:     plain per-lane sums, error-free FP32 pair ("double-word")
 *            merge across the warp and finalisation, no FP64 instruction
 *            (the default: FP64 is a small fraction of the FP32 rate on
 *            GB300).
 * Except in PLAIN, clip bounds and the sparsification threshold are rounded
 * outward-exact, so a float value is compared with the extended bound. */
#define SEP_PREC_PLAIN     0
#define SEP_PREC_KAHAN     1
#define SEP_PREC_FP64MERGE 2
#define SEP_PREC_DWORD     3

/* ---- opaque handles ---------------------------------------------------- */
typedef struct sep_ctx sep_ctx;
typedef struct sep_csr sep_csr;
typedef struct sep_calib sep_calib;
typedef struct sep_model sep_model;
typedef struct CUstream_st* sep_stream; /* identical to cudaStream_t */

/* ---- plain structs ----------------------------------------------------- */
/*
 * Flat detector normal to the beam (Section 2.2). Pixel (row, col) covers
 * [row, row+1) x [col, col+1) in pixel units; its centre is (row+0.5, col+0.5).
 */
typedef struct {
  int32_t rows, cols;        /* image shape, rows * cols <= SEP_MAX_PIXELS */
  double pixel_m[2];         /* pixel size (y, x) in metres */
  double dist_m;             /* sample-detector distance, metres */
  double center_px[2];       /* beam centre (x = column, y = row) in pixels */
  double wavelength_m;       /* metres (used by SEP_UNIT_Q_NM) */
  int32_t unit;              /* SEP_UNIT_* radial unit of the bins */
  int32_t nbins;             /* number of radial bins, 1 .. SEP_MAX_BINS */
  int32_t split;             /* 1: no splitting; 2: 2 x 2 sub-pixel centres;
                                0: exact area fractions (the area of the pixel
                                between the bin's two circles on the detector
                                plane over the pixel's area; per-entry weights,
                                a pixel may span at most 15 bins) */
  double range[2];           /* [lo, hi] in the unit; NaN = automatic (min/max over valid sub-pixel centres) */
} sep_geometry;

#define SEP_MAX_PIXELS (1 << 25)
#define SEP_MAX_BINS   32767
/* Frames per call of every call that takes device-resident frames or
 * per-frame device rows (their launches have one grid row per frame); a
 * larger n_frames returns SEP_ERR_ARG before any launch. sep_process_host
 * takes any count (its chunks must respect the limit), sep_veto up to 2^24. */
#define SEP_MAX_FRAMES 65535

/* Parameters of clipping and of the two consumers (Sections 2.4, 3, 4). */
typedef struct {
  int32_t n_iter;            /* maximum rejection steps (Section 2.4), >= 0 */
  float k_clip;              /* clip cut-off n of Eq. 19, > 0 */
  float k_pick;              /* sparsification cut-off (Section 3), >= 0 */
  int32_t patch;             /* peak patch side, odd, 1 .. 15 (Section 4) */
  int32_t min_count;         /* minimum kept pixels in the patch, >= 1 */
  int32_t precision;         /* SEP_PREC_* */
  int32_t surrogate;         /* 0: the first core of the clip kernel's replay is
                                placed from the first pass's moments; 1 .. 8:
                                from the prediction of the model attached to
                                the CSR (sep_csr_attach_model). The results are
                                those of the plain loop either way (the model
                                only changes how much of the row is replayed);
                                needs precision SEP_PREC_DWORD */
  int32_t cutoff;            /* SEP_CUTOFF_FIXED: every step clips at k_clip;
                                SEP_CUTOFF_CHAUVENET: the cut-off of each step is
                                Eq. 20's for the current set's size n,
                                sqrt(2 ln(n / sqrt(2 pi))), and a set of two
                                entries or fewer is not clipped (k_clip unused);
                                needs surrogate == 0 */
  int32_t error_model;       /* the deviation that clips and is reported
                                (Section 2.4.1): SEP_ERROR_AZIMUTHAL, the spread
                                of the bin's values (Eq. 13); SEP_ERROR_POISSON,
                                each pixel's variance is its value plus dark_var
                                (Eq. 3), propagated with squared coefficients
                                (Eq. 4, normalised as Eq. 13: sigma^2 =
                                sum c^2 (v + dark_var) / sum c^2); SEP_ERROR_HYBRID,
                                azimuthal clipping, Poisson deviation of the
                                final set. Poisson and hybrid: frames without a
                                norm, surrogate == 0 */
  float dark_var;            /* dark-noise variance sigma_dark^2 of Eq. 3, >= 0 */
  int32_t interpolate;       /* background of the two consumers (Sections 3, 4):
                                0: the pixel centre's bin, a pixel is kept iff
                                v > mu_b + k_pick sigma_b and peak records
                                subtract mu_b; 1: the smooth profile at the
                                pixel centre's radial value x (mean and
                                deviation interpolated linearly between the two
                                bin centres around x, the end bins' levels
                                beyond the outer centres, binary32), kept iff
                                v > mu(x) + k_pick sigma(x), and peak records
                                subtract mu(x) and propagate sigma(x). With 1
                                the batch calls mark kept pixels in a pass
                                after clipping instead of inside it */
} sep_params;

#define SEP_CUTOFF_FIXED     0
#define SEP_CUTOFF_CHAUVENET 1
#define SEP_ERROR_AZIMUTHAL  0
#define SEP_ERROR_POISSON    1
#define SEP_ERROR_HYBRID     2

/* One peak (Section 4). y, x: centroid in pixel units (row, column axes,
 * pixel centres at idx + 0.5); I: background-subtracted sum over the kept
 * patch pixels; sigma: propagated deviation sqrt(sum sigma_b^2). */
typedef struct {
  int32_t idx;               /* pixel index row * cols + col of the local maximum */
  float y, x, I, sigma;
  int32_t npix;              /* kept pixels in the patch */
} sep_peak;

/* ---- context ------------------------------------------------------------ */
const char* sep_version(void);

/* Create a context on CUDA device `device`. Allocates a 4-byte device status word. */
sep_status sep_ctx_create(int32_t device, sep_ctx** out);
void sep_ctx_destroy(sep_ctx* ctx);
/* Message of the last host-side failure on ctx (never NULL; "" if none). */
const char* sep_last_error(const sep_ctx* ctx);
/* Wait for `stream`, copy the device status word (SEP_DEV_* bits) to
 * *status_out and clear it. */
sep_status sep_get_device_status(sep_ctx* ctx, sep_stream stream, int32_t* status_out);

/* ---- integration matrix (Section 2.2) ------------------------------------ */
/*
 * Build the CSR matrix of coefficients c_{i,r} (the fraction of pixel i in
 * radial bin r, Section 2.2, measured by split x split sub-pixel centres, or
 * with split 0 the exact area fraction) on the host and upload it to the
 * context's device.
 *  mask_host: rows*cols bytes, nonzero = masked pixel (never used); may be NULL.
 *  norm_host: rows*cols floats, the normalisation of Eq. 1 (denominator);
 *             may be NULL (= 1 everywhere). Must be > 0 on valid pixels.
 * Rows of the matrix are bins. Within a row, entries are grouped by
 * coefficient (largest first, then weight-0 entries) and ordered by staging
 * position (see sep_csr_staging); the entries of one staging tile form a
 * run, padded (col -1, coefficient 0) to a multiple of 8 entries, so rows
 * and groups hold multiples of 8 entries. Every valid
 * pixel also gets its centre bin (the bin its threshold is taken from in
 * sparsification, Section 3); where that bin has no coefficient of the
 * pixel, an entry of weight 0 is added for it.
 * ctx may be NULL: the matrix is then built on the host only, for
 * inspection with sep_csr_info / sep_csr_export; compute calls need a matrix
 * built with a context (SEP_ERR_STATE otherwise).
 * Errors: SEP_ERR_ARG for invalid geometry; SEP_ERR_OOM.
 */
sep_status sep_build_csr(sep_ctx* ctx, const sep_geometry* geom, const uint8_t* mask_host,
                         const float* norm_host, sep_csr** out);
void sep_csr_destroy(sep_csr* csr);
/* Sizes: pixels, bins, nonzeros, largest row; range[2] as used. Any out pointer may be NULL. */
sep_status sep_csr_info(const sep_csr* csr, int64_t* npix, int32_t* nbins, int64_t* nnz,
                        int32_t* max_row, double* range);
/* Staging order: the order of the pixels with at least one matrix entry that
 * sorts the entries inside each coefficient group of a row (so one staging
 * tile writes consecutive slots of a bin's row). Pixels are grouped by tiles
 * of 64 rows x 64 columns (tiles in row-major order); inside a tile, by
 * centre bin, then radius of the pixel centre, then pixel index. perm_inv
 * [npos] receives the pixel of each position (may be NULL); *npos the number
 * of positions. (A frame's staged copy holds one value per matrix entry, in
 * row order: entry e's corrected pixel value at slot e.) */
sep_status sep_csr_staging(const sep_csr* csr, int32_t* perm_inv, int64_t* npos);
/* Interpolation table of the smooth background (Section 3; densification
 * and the consumers with interpolate): per pixel, the lower bin a [npix]
 * and the weight t [npix] (binary32, in [0, 1)) of the upper bin, so that
 * a profile p at the pixel centre is (1 - t) p[a] + t p[a+1]: u = (x - lo) /
 * (hi - lo) * nbins - 1/2 for the centre's radial value x, a = floor(u),
 * t = u - a rounded once; u <= 0 gives (0, 0) and u >= nbins - 1 gives
 * (nbins - 1, 0) (the end bins' levels). Masked pixels get (0, 0). Host
 * copies; either pointer may be NULL. */
sep_status sep_csr_interp(const sep_csr* csr, int32_t* lower_bin, float* weight);
/* Host copies for inspection (any pointer may be NULL):
 * rowptr [nbins+1], col [nnz] (-1 for padding), coef [nnz] (c_{i,r}; 0 for
 * padding and centre-only entries),
 * bin_of_pixel [npix] (-1 = masked), bin_centers [nbins]. */
sep_status sep_csr_export(const sep_csr* csr, int32_t* rowptr, int32_t* col, float* coef,
                          int32_t* bin_of_pixel, float* bin_centers);
/* Host-side check of an integration matrix in the layout sep_csr_export
 * writes (Section 2.2: one CSR row per radial bin), for matrices built or
 * edited outside the library. No device call; nothing is launched.
 *  rowptr [nbins+1]: rowptr[0] = 0, non-decreasing, rowptr[nbins] = nnz.
 *  col [nnz]: pixel index in [0, npix), or -1 for a padding slot.
 *  coef [nnz]: finite, in [0, 1]; 0 on padding slots; the coefficients of
 *      one pixel over all bins sum to at most 1 (its area, up to 1e-6).
 *  bin_of_pixel [npix] (may be NULL): in [-1, nbins).
 *  calib_npix: the pixel count of the calibration to be used with the
 *      matrix (must equal npix), or -1 for no calibration.
 *  msg [msg_len] (may be NULL): receives the first violation, or "".
 * Returns SEP_OK, or SEP_ERR_ARG at the first violation (non-monotone
 * row pointer, column, coefficient or bin out of range, calibration of
 * another size). */
sep_status sep_csr_validate(const int32_t* rowptr, const int32_t* col, const float* coef,
                            const int32_t* bin_of_pixel, int32_t nbins, int64_t nnz, int64_t npix,
                            int64_t calib_npix, char* msg, int32_t msg_len);
/* The same checks on a built matrix handle (its host copy, plus the tables
 * the kernels follow: class ends, centre entries, staging scatter lists)
 * and, when calib is not NULL, that the calibration covers the detector
 * and belongs to the matrix's context. sep_build_csr runs the matrix checks
 * itself before any upload. SEP_OK or SEP_ERR_ARG / SEP_ERR_STATE (reason
 * in sep_last_error of the matrix's context). Host only. */
sep_status sep_csr_check(const sep_csr* csr, const sep_calib* calib);

/* ---- detector calibration (Section 1.2) ---------------------------------- */
/*
 * Upload per-pixel pedestals and gains of the three Jungfrau gain levels,
 * plane-major: ped_host[g * npix + i], gain_host[g * npix + i], g = 0, 1, 2.
 * A raw word with gain code 0 uses level 0, code 1 level 1, codes 2 and 3
 * level 2. The corrected value is RN32(RN32(adc - ped) / gain).
 */
sep_status sep_calib_create(sep_ctx* ctx, const sep_csr* csr, const float* ped_host,
                            const float* gain_host, sep_calib** out);
void sep_calib_destroy(sep_calib* calib);

/* ---- compute calls -------------------------------------------------------- */
/*
 * Integrate and sigma-clip n_frames frames (Eqs. 2, 8-13, 19; Section 2.4).
 *  frames_dev: [n_frames][npix] of dtype (uint16 raw words need calib,
 *              float32 ignores calib).
 *  Outputs (device, [n_frames][nbins]): mean_dev (clipped weighted mean),
 *  sigma_dev (clipped deviation sqrt(VV / OmegaOmega), Eq. 13), count_dev
 *  (entries of nonzero weight in the final set).
 *  bounds_dev: optional [n_frames][nbins][2] float32 interval [L, H] such
 *  that the final set is every entry with L <= value <= H; may be NULL.
 *  iters_dev: optional [n_frames][nbins] int32 rejection steps taken; may be NULL.
 */
sep_status sep_integrate_clip(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib,
                              const void* frames_dev, int32_t dtype, int32_t n_frames,
                              const sep_params* params, float* mean_dev, float* sigma_dev,
                              int32_t* count_dev, float* bounds_dev, int32_t* iters_dev,
                              sep_stream stream);

/*
 * Sparsify (Section 3): keep valid pixel i when value_i > mean_b + k_pick sigma_b,
 * b = centre bin of i (with params->interpolate: the profile interpolated at
 * the pixel centre, mean(x_i) + k_pick sigma(x_i); the threshold is that sum
 * rounded down to binary32). Writes, per frame, the first `capacity` kept pixels in
 * ascending index order: idx_dev [n_frames][capacity] (int32) and val_dev
 * [n_frames][capacity] (float32 value), and the true count n_kept_dev
 * [n_frames]. A count above capacity sets SEP_DEV_CAPACITY.
 */
sep_status sep_sparsify(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib,
                        const void* frames_dev, int32_t dtype, int32_t n_frames,
                        const sep_params* params, const float* mean_dev, const float* sigma_dev,
                        int32_t* idx_dev, float* val_dev, int64_t capacity, int32_t* n_kept_dev,
                        sep_stream stream);

/*
 * Peak picking (Section 4) over the kept pixels given by a previous
 * sep_sparsify (idx_dev, n_kept_dev, kept_capacity). A kept pixel is a peak
 * when it is the maximum of its patch (ties: the lowest index wins) and at
 * least min_count patch pixels are kept. Its record: I = sum of
 * (value_j - background_j) over the kept patch pixels j, the centroid of
 * those weights, sigma = sqrt(sum of deviation_j^2), with background and
 * deviation the pixel's bin levels (params->interpolate: the profile at the
 * pixel centre). Writes the first `capacity` peaks per frame in ascending
 * index order to peaks_dev [n_frames][capacity] and the true count to
 * n_peaks_dev [n_frames].
 */
sep_status sep_peakfind(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib,
                        const void* frames_dev, int32_t dtype, int32_t n_frames,
                        const sep_params* params, const float* mean_dev, const float* sigma_dev,
                        const int32_t* idx_dev, const int32_t* n_kept_dev, int64_t kept_capacity,
                        sep_peak* peaks_dev, int64_t capacity, int32_t* n_peaks_dev,
                        sep_stream stream);

/*
 * Densification (Section 3, "Densification / Decompression"): rebuild dense
 * frames from their sparse form. Every pixel with a centre bin b gets the
 * bin's background level m_i = mean_dev[f][b] (s_i = sigma_dev[f][b]), or with
 * interpolate != 0 the smooth profile: the linear interpolation of the bins'
 * levels at the pixel centre's radial value between the two nearest bin
 * centres (end bins' levels beyond the outer centres), in binary32:
 * m_i = RN(RN(RN(1 - t_i) mean_a) + RN(t_i mean_(a+1))), s_i likewise;
 * when noise_dev is given (standard normal deviates z, float32
 * [n_frames][npix], drawn by the caller) the pixel gets RN32(m_i + RN32(s_i *
 * z_i)) instead (the noisy background some reduction programs need); then
 * the first min(n_kept[f], kept_capacity)
 * kept pixels of the frame (idx_dev / val_dev [n_frames][kept_capacity], as
 * sep_sparsify writes them; indices outside the detector are skipped) get
 * their recorded values back. Pixels without a bin (masked) get `fill`.
 * mean/sigma: [n_frames][nbins] float32 (sigma may be NULL without noise).
 * out_dev: float32 [n_frames][npix], caller-owned. No scratch is used.
 */
sep_status sep_densify(sep_ctx* ctx, const sep_csr* csr, int32_t n_frames, const float* mean_dev,
                       const float* sigma_dev, const int32_t* idx_dev, const float* val_dev,
                       int64_t kept_capacity, const int32_t* n_kept_dev, const float* noise_dev, float fill,
                       int32_t interpolate, float* out_dev, sep_stream stream);

/*
 * Veto (Section 4, "Peak count as veto algorithm"): frame f passes when it
 * has at least min_peaks peaks (n_peaks_dev[f] >= min_peaks; frames with fewer
 * are discarded). Writes the passing frames' indices in ascending order to
 * frame_list_dev [n_frames] (int32; the first *n_pass_dev entries are
 * meaningful) and their count to n_pass_dev (int32 [1]). One CTA; n_frames
 * <= 2^24. min_peaks >= 0.
 */
sep_status sep_veto(sep_ctx* ctx, int32_t n_frames, const int32_t* n_peaks_dev, int32_t min_peaks,
                    int32_t* frame_list_dev, int32_t* n_pass_dev, sep_stream stream);

/*
 * Frame-drop compaction after sep_veto: row j of dst_dev becomes row
 * frame_list_dev[j] of src_dev for j < *n_pass_dev (rows of row_bytes bytes,
 * a multiple of 4; n_frames rows at most); rows of dst_dev past the count are
 * left as they were. Works for any per-frame output array (mean, sigma,
 * kept lists, peak records, ...). src and dst must not overlap.
 */
sep_status sep_compact_frames(sep_ctx* ctx, int32_t n_frames, const int32_t* frame_list_dev,
                              const int32_t* n_pass_dev, int64_t row_bytes, const void* src_dev, void* dst_dev,
                              sep_stream stream);

/*
 * The whole path on a batch in one call: integrate + clip, sparsify and peak
 * picking, with the kept-pixel map passed between the steps on the device.
 * Outputs as in the three calls above. The launch sequence is captured once
 * per (csr, calib, dtype, n_frames, capacities, params) into a CUDA graph and
 * replayed on later calls with the same shapes (use_graph = 1).
 */
sep_status sep_process_batch(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib,
                             const void* frames_dev, int32_t dtype, int32_t n_frames,
                             const sep_params* params, float* mean_dev, float* sigma_dev,
                             int32_t* count_dev, int32_t* idx_dev, float* val_dev,
                             int64_t kept_capacity, int32_t* n_kept_dev, sep_peak* peaks_dev,
                             int64_t peak_capacity, int32_t* n_peaks_dev, int32_t use_graph,
                             sep_stream stream);

/* One frame of a mixed batch: its detector (index into the csr / calib
 * arrays), its dtype (all frames of one detector share it) and its device
 * address. */
typedef struct {
  int32_t det;
  int32_t dtype;
  const void* frame_dev;
} sep_frame_desc;

/*
 * The whole path on a stream of frames from up to 4 detectors of different
 * sizes (their own matrices, calibrations and clip schedules) in one call:
 * each detector's frames run as one parallel branch of a single captured
 * CUDA graph (use_graph = 1), replayed for the same descriptors and outputs.
 *  frames: host array [n_frames] of descriptors, in stream order.
 *  mean/sigma/count_dev: flat per-bin outputs, frame g's nbins values at
 *  row_off[g]; row_off (host, [n_frames + 1], may be NULL) receives the
 *  offsets (prefix sums of the frames' bin counts).
 *  idx/val_dev [n_frames][kept_capacity], n_kept_dev [n_frames],
 *  peaks_dev [n_frames][peak_capacity], n_peaks_dev [n_frames]: as in
 *  sep_process_batch, rows in stream order.
 * Blocks the host until the previous call on `stream` has read its
 * descriptor table (a few bytes per frame).
 */
sep_status sep_process_mixed(sep_ctx* ctx, int32_t n_det, sep_csr* const* csrs,
                             const sep_calib* const* calibs, const sep_frame_desc* frames,
                             int32_t n_frames, const sep_params* params, float* mean_dev,
                             float* sigma_dev, int32_t* count_dev, int64_t* row_off, int32_t* idx_dev,
                             float* val_dev, int64_t kept_capacity, int32_t* n_kept_dev,
                             sep_peak* peaks_dev, int64_t peak_capacity, int32_t* n_peaks_dev,
                             int32_t use_graph, sep_stream stream);

/*
 * Schedule of the integrate + clip kernel for one matrix (a tuning choice,
 * results do not depend on it): bins are grouped by row length into
 * n_classes size classes (1..4; class i holds rows with thresholds[i-1] < n
 * <= thresholds[i], ascending, n_classes - 1 thresholds), each launched with
 * tpb[i] threads per block (64, 128 or 256) and shared memory for its own
 * longest row; classes run as parallel branches. Default: one class, 256.
 */
sep_status sep_csr_set_plan(sep_ctx* ctx, sep_csr* csr, int32_t n_classes, const int32_t* thresholds,
                            const int32_t* tpb);
/* Current plan: *n_classes, thresholds[n_classes-1], tpb[n_classes] (arrays of 4). */
sep_status sep_csr_get_plan(const sep_csr* csr, int32_t* n_classes, int32_t* thresholds, int32_t* tpb);
/*
 * Time candidate plans (single class at 64/128/256 threads; two classes split
 * at 1024/2048/4096/8192 entries with every block-size pair; three classes
 * split at 4096/8192, 6144/10240 or 4096/10240 entries with four block-size
 * triples) on a sample
 * batch of device frames with sep_integrate_clip's work, keep the fastest on
 * csr and report its time per call in *best_ms (may be NULL). cache_path
 * (may be NULL): a text file keyed by detector shape, matrix, dtype,
 * precision and device name; a plan found there is applied without timing,
 * a new one is appended. Allocates and frees a temporary output buffer.
 */
sep_status sep_autotune(sep_ctx* ctx, sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                        int32_t dtype, int32_t n_frames, const sep_params* params, const char* cache_path,
                        float* best_ms, sep_stream stream);

/* ---- learned surrogate of the clip iteration ------------------------------ */
/*
 * A small network (no counterpart in the paper) predicts a bin's clipped mean
 * and deviation, i.e. its final clip interval, from statistics of a sample of
 * its entries. The clip kernel replays the loop of Eq. 19 exactly on the sums
 * of a core interval that lies inside every interval the loop visits, plus
 * the entries outside it; the prediction places that core (half a predicted
 * deviation inside the predicted final interval), so a good prediction spares
 * the re-placements and rescans of the row that the plain placement (inside
 * the first interval) needs, and a poor one costs a rescan. The loop itself,
 * and so every result, is the plain method's: the plain loop judges every
 * step. Network: SEP_MLP_IN features -> 64 -> GELU -> 64 -> GELU -> 2,
 * GELU exact (x Phi(x)), weights stored BF16 for every forward / backward,
 * FP32 master copy and FP32 accumulation. Parameter layout (floats):
 * W1 [64][20], b1 [64], W2 [64][64], b2 [64], W3 [2][64], b3 [2].
 * Normalisation block: feature mean [20], feature deviation [20], target
 * mean [2], target deviation [2] (used only by the clip kernel's inference;
 * sep_mlp_* and sep_surrogate_train work on already normalised data).
 */
#define SEP_MLP_IN 20
#define SEP_MLP_HIDDEN 64
#define SEP_MLP_OUT 2
#define SEP_MLP_PARAMS 5634
#define SEP_MLP_NORM 44

typedef struct {
  int32_t epochs;   /* passes over the samples, >= 1 */
  int32_t batch;    /* samples per Adam step, >= 64 */
  float lr;         /* Adam learning rate, > 0 */
  int32_t pad;
  uint64_t seed;    /* visiting order */
} sep_train_cfg;

/* New model with He-uniform weights from `seed`, zero biases, identity normalisation. */
sep_status sep_model_create(sep_ctx* ctx, uint64_t seed, sep_model** out);
void sep_model_destroy(sep_model* model);
/* Copy the parameters out to get_host and / or in from set_host (either may be NULL), [SEP_MLP_PARAMS]. */
sep_status sep_model_params(sep_model* model, float* get_host, const float* set_host);
/* Same for the normalisation block [SEP_MLP_NORM]; deviations must be > 0. */
sep_status sep_model_norm(sep_model* model, float* get_host, const float* set_host);
/* y_dev [n][2] = network(x_dev [n][20]) on device memory. */
sep_status sep_mlp_forward(sep_model* model, const float* x_dev, int64_t n, float* y_dev, sep_stream stream);
/* Loss L = mean over n samples of the summed squared error against t_dev [n][2]
 * into *loss_dev, and dL/dparams into grad_dev [SEP_MLP_PARAMS] (device). */
sep_status sep_mlp_loss_grad(sep_model* model, const float* x_dev, const float* t_dev, int64_t n,
                             float* grad_dev, float* loss_dev, sep_stream stream);
/* Adam (0.9, 0.999, 1e-8) over n samples in a pseudo-random order; the
 * last epoch's mean loss goes to *final_loss (may be NULL). Synchronises. */
sep_status sep_surrogate_train(sep_model* model, const float* x_dev, const float* t_dev, int64_t n,
                               const sep_train_cfg* cfg, float* final_loss, sep_stream stream);
/* Attach a model to a CSR (NULL detaches). The CSR keeps the pointer, not a
 * copy: the model must outlive its use, and later training of the model is
 * seen by later launches. Calls with params->surrogate > 0 then place each
 * bin's first core from the model's prediction: with the sample mean m1 and
 * deviation s1 of the bin (the features below), mu^ = m1 + s1 y0 and sd^ =
 * s1 exp(y1) (y de-normalised by the target block); the core is
 * [mu^ - k sd^ + sd^ / 2, mu^ + k sd^ - sd^ / 2]. Every result (mean, sigma,
 * count, bounds, iterations, kept pixels) is the plain loop's, whatever the
 * prediction; the sums may be taken in another order. */
sep_status sep_csr_attach_model(sep_csr* csr, const sep_model* model);

/* The whole path from host memory to host memory, pipelined: the batch is
 * cut into chunks of chunk_frames frames (0 = 64); chunk c+1 is copied in
 * while chunk c is processed (sep_process_batch on device buffers owned by
 * the context, three chunk slots) and chunk c-1's results are copied out,
 * on three streams.
 * Host arrays are as sep_process_batch's device arrays (frames_host
 * [n_frames][npix], mean/sigma/count [n_frames][nbins], idx/val
 * [n_frames][kept_capacity], n_kept [n_frames], peaks [n_frames][peak_capacity],
 * n_peaks [n_frames]); they should be pinned (cudaHostAlloc / torch
 * pin_memory) for the copies to overlap, and must stay valid until `stream`
 * completes: the call returns once everything is enqueued, with the work
 * ordered before any later work on `stream`. frames_host must hold its data
 * when the call is made: the copy-in does not wait for earlier work on
 * `stream`, so that consecutive calls overlap. */
sep_status sep_process_host(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_host,
                            int32_t dtype, int32_t n_frames, const sep_params* params, float* mean_host,
                            float* sigma_host, int32_t* count_host, int32_t* idx_host, float* val_host,
                            int64_t kept_capacity, int32_t* n_kept_host, sep_peak* peaks_host,
                            int64_t peak_capacity, int32_t* n_peaks_host, int32_t chunk_frames, sep_stream stream);

/* Corrected frames (Section 1.2 and Eq. 1): out_dev [n_frames][npix] float32
 * receives RN32(RN32(adc - ped[g]) / gain[g]) (raw Jungfrau words, dtype
 * SEP_DTYPE_U16_JF) or the float32 input, divided by the norm when the
 * matrix has one, for every pixel the matrix uses; pixels it does not use
 * (masked, outside the radial range) receive NaN. These are the values the
 * integration reads. Uses the context's staging buffer. */
sep_status sep_correct(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                       int32_t dtype, int32_t n_frames, float* out_dev, sep_stream stream);

/* Plain clip (params->surrogate must be 0) that also records, per frame and
 * bin, the surrogate's input features feat_dev [n_frames][nbins][SEP_MLP_IN]
 * and its training targets target_dev [n_frames][nbins][2] =
 * ((mu - m1) / s1, log(sd / s1)) of the clipped result (NaN where the bin has
 * fewer than 2 entries in the final set, a zero deviation, or s1 = 0).
 * The first features are taken on a sample of the bin's row: every step-th
 * group of 4 consecutive entries of each coefficient class (step 4 for rows
 * of 2048 entries or more, 2 from 512, else 1); m1 and s1 are the sample's
 * mean and deviation (Eqs. 12-13, FP32). Features: 0 log(step n) / 8 (n:
 * the sample's finite entries of weight != 0), 1 Omega / n over the sample,
 * 2 clamp(m1 / s1, -20, 20) / 4. The rest come from a sketch of at most 128
 * of the row's weighted entries (element s = 0 .. 127 is entry s when the
 * G groups of 4 before the weight-0 carriers hold at most 128 entries, else
 * entry 4 floor(s G / 128) + s mod 4; non-finite values left out): 3 the
 * sketch's fraction with v >= m1 + 4 s1, 4 .. 19 its values at ranks
 * floor((j + 1/2) n' / 16) of n' in ascending order, as z = (v - m1) / s1
 * clamped to [-4, 12]. */
sep_status sep_surrogate_record(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                                int32_t dtype, int32_t n_frames, const sep_params* params, float* mean_dev,
                                float* sigma_dev, int32_t* count_dev, float* feat_dev, float* target_dev,
                                sep_stream stream);

/* Training set from recorded rows: keeps the rows whose features and targets
 * are finite (order preserved), computes the normalisation block over them
 * (mean and population deviation of each feature and target; a deviation
 * below 1e-6 becomes 1) into norm_host [SEP_MLP_NORM], and writes the kept
 * rows normalised to x_dev [n_valid][20], t_dev [n_valid][2] (room for n
 * rows each). Synchronises the stream. */
sep_status sep_surrogate_prepare(sep_ctx* ctx, const float* feat_dev, const float* target_dev, int64_t n,
                                 float* x_dev, float* t_dev, float* norm_host, int64_t* n_valid, sep_stream stream);

/* Of the bins the surrogate placed: how many kept the predicted core to the
 * end of their loop (accepted) and how many had to re-place it inside a later
 * interval and rescan the row (fell_back), summed over every call since the
 * last reset. Synchronises. */
sep_status sep_surrogate_stats(sep_ctx* ctx, uint64_t* accepted, uint64_t* fell_back, int32_t reset,
                               sep_stream stream);

/* Counters of the clip kernel's tail replay (diagnostics; the method is
 * unchanged by them). With collection enabled, every later integrate-clip,
 * batch and mixed call adds to SEP_CLIP_STATS counters held by the context:
 *   [0] bin-frame items, [1] core scans (pass B), [2] items whose tail slots
 *   overflowed (their remaining steps ran as full passes), [3] replay steps,
 *   [4] tail entries listed (summed over core scans), [5] items whose
 *   kept-pixel marks came from the tail alone, [6] full passes,
 *   [7] reserved (0).
 * enable: 1 collect, 0 stop, -1 leave as is (collection costs a few atomics
 * per block). counts: NULL or SEP_CLIP_STATS values written on return.
 * reset: nonzero zeroes the counters after reading. Synchronises `stream`
 * when counts or reset are requested. SEP_ERR_ARG for a NULL context or
 * enable outside {-1, 0, 1}. */
#define SEP_CLIP_STATS 8
sep_status sep_clip_stats(sep_ctx* ctx, int32_t enable, uint64_t* counts, int32_t reset, sep_stream stream);

/* Checkpoint: one JSON header line, then float32 parameters, normalisation,
 * Adam moments. */
sep_status sep_model_save(const sep_model* model, const char* path);
sep_status sep_model_load(sep_ctx* ctx, const char* path, sep_model** out);

/*
 * sep_sparsify with no allocation during the call (the paper has no
 * counterpart; this is an interface for callers, not part of the method).
 * sep_sparsify grows context-owned scratch with cudaMalloc when a batch needs
 * more; callers that must not allocate at call time (real-time acquisition
 * threads, processes whose device memory is fixed after start-up) use this
 * variant instead. Its scratch is one static 16 MiB device array in the
 * library, which every GPU that loads the library holds until exit.
 * Arguments, their checks (the same refusals), outputs and results are those
 * of sep_sparsify.
 *  - Limit: n_frames * (bitmap bytes ceil(npix/32)*4 rounded up to 32, plus
 *    4 * nbins, plus 4 per 8192 bitmap words) must fit 16 MiB (about 28
 *    Jungfrau-4M frames, about 1900 frames of 256 x 256); larger batches
 *    return SEP_ERR_ARG before any launch (split the batch).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, no allocation).
 *  - All calls share the array, which keeps the last call's contents; calls
 *    that overlap on the GPU (other streams or host threads) race on it.
 */
sep_status sep_sparsify_noalloc(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib,
                                const void* frames_dev, int32_t dtype, int32_t n_frames,
                                const sep_params* params, const float* mean_dev,
                                const float* sigma_dev, int32_t* idx_dev, float* val_dev,
                                int64_t capacity, int32_t* n_kept_dev, sep_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* SEP_H_ */
