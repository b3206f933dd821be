/*
 * spd.h -- C ABI of the GB300 single-pulse-detection library (libspd.so).
 *
 * Method: Adamek & Armour, "Single Pulse Detection Algorithms for Real-time
 * Fast Radio Burst Searches using GPUs" (arXiv:1910.08324).  The library
 * searches many dedispersed time series (one row per DM trial) with boxcar
 * filters (Eq. boxcar), normalises every boxcar to an SNR (Eq. SNRlong with the
 * white-noise statistics of Eq. whitenoise), keeps per start sample the
 * highest SNR and the width that produced it (Eq. MSD03, all iterations
 * combined), and selects candidates by threshold and peak finding (Sec. 4.5).
 * Width grids: every width up to L_max (the ideal search of Sec. 3.1), BoxDIT
 * (Alg. 1, Sec. 3.1) and IGRID (Sec. 3.2, Eq. boxcarsize, Table 1).
 *
 * Conventions
 *   - All device pointers belong to the caller.  The library never allocates
 *     device memory: scratch space is passed in as a workspace.  A plan owns
 *     host memory only.
 *   - Layout: row r of a [ndm][ld] array starts at element r*ld; samples of a
 *     row are contiguous in time.  Inputs and outputs share the row stride ld.
 *   - A boxcar is indexed by its first sample s (Eq. boxcar looks forward).
 *     Width L is evaluated at s iff s is a multiple of its boxcar separation
 *     L_s (Sec. 2.2.1) and s + L <= nt; nothing beyond a row is read or
 *     padded into a sum.  Width 1 is in every grid, so every start s < nt
 *     has a result.
 *   - Width indices refer to the plan's ascending width table
 *     (spd_plan_widths); ties in SNR go to the smallest width.
 *   - Calls taking a stream are asynchronous and never synchronise unless
 *     stated.  Validation errors are returned synchronously, before any
 *     work is queued.  Launch errors are returned as SPD_ERR_CUDA; errors of
 *     earlier asynchronous work surface in a later call or in
 *     spd_sync_status().  Nothing aborts, traps or prints.
 *   - Thread safety: a plan is read-only after creation and may be used from
 *     several host threads and streams at once.
 */
#ifndef SPD_H
#define SPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPD_VERSION_MAJOR 0
#define SPD_VERSION_MINOR 1

/* A CUDA stream handle (cudaStream_t).  NULL is the legacy default stream. */
typedef struct CUstream_st *spd_stream_t;

typedef enum spd_status {
  SPD_OK = 0,
  SPD_ERR_INVALID_ARG = 1,         /* a NULL pointer, bad size, bad enum, misaligned buffer */
  SPD_ERR_UNSUPPORTED = 2,         /* valid request this build does not implement */
  SPD_ERR_CUDA = 3,                /* a CUDA runtime call or kernel launch failed */
  SPD_ERR_WORKSPACE_TOO_SMALL = 4, /* ws_bytes below spd_workspace_size() */
  SPD_ERR_BUFFER_TOO_SMALL = 5,    /* a caller buffer (e.g. the width table) is too small */
  SPD_ERR_TIMEOUT = 6,             /* a bounded device-side wait gave up */
  SPD_ERR_HOST_ALLOC = 7           /* host memory for the plan could not be allocated */
} spd_status;

typedef enum spd_algo {
  SPD_ALGO_EXHAUSTIVE = 0, /* every width 1..s_end at every sample (ideal search, Sec. 3.1) */
  SPD_ALGO_BOXDIT = 1,     /* BoxDIT, Alg. 1 with L^i_max = boxdit_lmax for all i, D = 2 */
  SPD_ALGO_IGRID = 2       /* IGRID IG(d) with P layers per step (Sec. 3.2); d = 0, P = 1 is DIT (Alg. 3) */
} spd_algo;

/* Input sample types.  Every type is converted to float32 on load (exactly:
 * each value of these types is a float32 value) and summed in float32; mu and
 * sigma of spd_noise are in the units of the stored values. */
typedef enum spd_dtype {
  SPD_F32 = 0, /* 32-bit IEEE float samples (the paper's input type, Sec. 4) */
  SPD_F16 = 1, /* 16-bit IEEE half floats */
  SPD_BF16 = 2,/* bfloat16 (the high 16 bits of a float32) */
  SPD_U8 = 3   /* unsigned 8-bit integers (e.g. digitised filterbank data) */
} spd_dtype;

/*
 * Plan description (Sec. 2.2.1: a search is characterised by its width set and
 * the boxcar separation of every width).
 *   algo          spd_algo
 *   dtype         spd_dtype of the input samples
 *   s_end         widest pulse searched, S_end (Sec. 3).  The last width of the
 *                 grid is the first one >= s_end ("nearest longer", L_end).
 *                 For SPD_ALGO_EXHAUSTIVE it is L_max itself (1..4096).
 *                 L_end must not exceed 32768.
 *   boxdit_lmax   BoxDIT: widths computed per iteration, L^i_max (Alg. 1), the
 *                 same for every iteration: any even value 2..256 (Sec. 3.1
 *                 requires only divisibility by D = 2).  8, 16 and 32 (BD-8/16/32
 *                 of Sec. 4) run on dedicated streaming kernels, every other
 *                 value on the general BoxDIT kernel; spd_plan_create_boxdit
 *                 takes one value per iteration.
 *   igrid_depth   IGRID: depth d of Eq. boxcarsize, 0..3.
 *   igrid_layers  IGRID: layers per step P (power of two, 2^d <= P, P <= 2^(d+1));
 *                 IG(1), IG(2), IG(3) of Sec. 3.2.1 use 4, 8, 16; DIT uses d=0, P=1.
 *   ndm, nt, ld   rows (DM trials), samples per row, row stride in elements
 *                 (ld >= nt).  ndm >= 1, nt >= 1.
 */
typedef struct spd_plan_desc {
  int32_t algo;
  int32_t dtype;
  int32_t s_end;
  int32_t boxdit_lmax;
  int32_t igrid_depth;
  int32_t igrid_layers;
  int64_t ndm;
  int64_t nt;
  int64_t ld;
} spd_plan_desc;

/*
 * Noise statistics used for the SNR of Eq. SNRlong, (X_L - mu_L) / sigma_L.
 *   mode 0 (white): mu[ndm], sigma[ndm] are the mean and standard deviation of
 *                   each row's samples; a width-L boxcar uses mu_L = L*mu and
 *                   sigma_L = sqrt(L)*sigma (Eq. whitenoise).
 *   mode 1 (table): mu[ndm][n_widths], sigma[ndm][n_widths] (row-major) give
 *                   mu_L and sigma_L of every row for every width of the plan,
 *                   in the order of spd_plan_widths (index 0 is width 1).  For
 *                   noise that is not white, e.g. red noise or statistics
 *                   measured at several decimations (Sec. 4.5).
 * Both pointers are device pointers to float32, 4-byte aligned; every sigma
 * must be finite and > 0 and every mu finite (not checked: other values give
 * meaningless SNRs, no error).
 */
typedef struct spd_noise {
  int32_t mode;
  const float *mu;
  const float *sigma;
} spd_noise;

/* One detection (Sec. 4.5 candidate list): row, start sample, SNR and width. */
typedef struct spd_candidate {
  int32_t row;       /* DM-trial row */
  int32_t width_idx; /* index into the plan's width table */
  int64_t start;     /* first sample of the boxcar (centre = start + width/2) */
  float snr;         /* Y[row][start] */
  int32_t width;     /* the width itself, in samples */
} spd_candidate;

typedef struct spd_plan spd_plan;

/* Human-readable text for a status code (static storage, never NULL). */
const char *spd_status_string(spd_status status);

/* "major.minor" of this library (static storage). */
const char *spd_version(void);

/*
 * Build a plan: validates the description and derives the width grid of the
 * chosen algorithm (Sec. 3.1 Alg. 1 width formula; Sec. 3.2 Eq. boxcarsize and
 * Table 1).  Host only: no device work, no device memory.
 * Errors: SPD_ERR_INVALID_ARG for a NULL pointer or any parameter outside the
 * ranges documented in spd_plan_desc; SPD_ERR_UNSUPPORTED for a plan whose
 * kernel would exceed the device limits (shared memory, grid size);
 * SPD_ERR_HOST_ALLOC.  *out is NULL on error.
 */
spd_status spd_plan_create(const spd_plan_desc *desc, spd_plan **out);

/*
 * Build a BoxDIT plan with a maximum width per iteration (Alg. 1; Sec. 3.1 lets
 * L^i_max change from iteration to iteration, to trade signal loss between
 * pulse widths).  Iteration i uses lmax[i]; iterations past n_lmax use
 * lmax[n_lmax - 1].  Iteration i computes the widths L^{i-1}_MAX + 2^i m,
 * m = 1..L^i_max, at every 2^i-th start, with L^i_MAX = L^{i-1}_MAX + 2^i L^i_max.
 *   lmax     host array of n_lmax even values, each 2..256 (read during the call)
 *   n_lmax   1..24
 *   n_iter   0: iterate up to the first width >= desc->s_end (nearest longer,
 *            as spd_plan_create); 1..24: exactly n_iter full iterations
 *            (desc->s_end is then ignored; the paper counts BD-8's iterations
 *            this way in Sec. 4)
 * desc supplies dtype, ndm, nt, ld (and s_end when n_iter is 0); its algo and
 * boxdit_lmax are ignored.  The widest width must not exceed 32768 and the grid
 * must have at most 512 widths.  A plan whose L^i_max are all 8, all 16 or all
 * 32 runs on the BD-K streaming kernels, any other on the general BoxDIT
 * kernel (tiles of 2048 to 8192 starts, see spd_plan_set_segment).  Host only.
 * Errors as spd_plan_create.
 */
spd_status spd_plan_create_boxdit(const spd_plan_desc *desc, const int32_t *lmax, int32_t n_lmax,
                                  int32_t n_iter, spd_plan **out);

/*
 * Build a plan over an explicit grid: Sec. 2.2 characterises a search by its
 * set of boxcar widths and the boxcar separation L_s of each width; here both
 * are given as lists, widths[i] searched at the starts that are multiples of
 * seps[i].  widths strictly increasing, 1 <= widths[i] <= 4096,
 * widths[0] == 1 with seps[0] == 1 (every start has a value); seps powers of
 * two <= 4096; 1 <= n_widths <= 512.  desc supplies dtype, ndm, nt and ld (its
 * algorithm fields are ignored).  Searched like the exhaustive grid, widths
 * outside the set skipped: width index i of snr / width_idx is widths[i].  Host
 * only.  SPD_ERR_INVALID_ARG for a set or shape that breaks these rules.
 */
spd_status spd_plan_create_grid(const spd_plan_desc *desc, const int32_t *widths, const int32_t *seps,
                                int32_t n_widths, spd_plan **out);
/* Release a plan (NULL is accepted).  No device synchronisation. */
spd_status spd_plan_destroy(spd_plan *plan);

/*
 * The plan's width table in ascending order: widths[i] (samples) and the
 * boxcar separation seps[i] (Sec. 2.2.1).  Either array may be NULL to query
 * only *n.  SPD_ERR_BUFFER_TOO_SMALL if cap < *n (nothing is written then).
 */
spd_status spd_plan_widths(const spd_plan *plan, int32_t *widths, int32_t *seps,
                           int32_t cap, int32_t *n);

/*
 * Bytes of device workspace the plan needs for spd_execute, spd_candidates,
 * spd_search and spd_noise_stats (256-byte aligned base required).
 */
spd_status spd_workspace_size(const spd_plan *plan, size_t *bytes);

/*
 * The search (Eq. boxcar, Eq. SNRlong, Eq. MSD03).  For every row r and every
 * start s in [0, nt):
 *   snr[r*ld + s]       = max over eligible widths L of (X_L[s] - L mu_r)/(sqrt(L) sigma_r)
 *   width_idx[r*ld + s] = index of the smallest width reaching that maximum
 * where X_L[s] is the sum of the L samples starting at s.  Width 1 is in every
 * grid, so every s has a value.  Samples at s >= nt of a row (the ld - nt
 * padding) are neither read nor written.
 *   d_x         device, [ndm][ld] samples of plan dtype, aligned to the sample
 *               size (a 16-byte aligned base with ld * sample size a multiple
 *               of 16 enables vector loads)
 *   noise       host struct holding device pointers (white or table mode)
 *   d_snr       device, [ndm][ld] float32 output
 *   d_width_idx device, [ndm][ld] uint16 output
 *   d_ws        device workspace of at least spd_workspace_size() bytes, or NULL
 *               if that size is 0; 256-byte aligned.  On return it holds the
 *               maximum SNR of every tile of every row (used by spd_search).
 *   stream      stream all work is queued on
 * Errors: SPD_ERR_INVALID_ARG (NULL or misaligned pointers, noise mode not 0
 * or 1), SPD_ERR_WORKSPACE_TOO_SMALL, SPD_ERR_CUDA (launch failure).
 * Outputs are only valid once the stream has reached this work.
 */
spd_status spd_execute(const spd_plan *plan, const void *d_x, const spd_noise *noise,
                       float *d_snr, uint16_t *d_width_idx, void *d_ws, size_t ws_bytes,
                       spd_stream_t stream);

/*
 * Candidate selection on the outputs of spd_execute (the peak-finding step of
 * Sec. 4.5, which the paper does not define).  Start s of row r is a candidate
 * iff snr[s] >= threshold, snr[s] > snr[s'] for s - R <= s' < s and
 * snr[s] >= snr[s'] for s < s' <= s + R (s' inside [0, nt)), R = peak_radius
 * (0 = plain threshold, at most 64).  Records are written in (row, start)
 * order; the first min(cap, total) are stored in d_out and the total count is
 * stored in *d_count (device int64).  When *d_count > cap the list is
 * truncated; the call itself still returns SPD_OK (it does not synchronise):
 * spd_candidates_status reports the overflow as SPD_ERR_BUFFER_TOO_SMALL.
 *   d_snr, d_width_idx  device outputs of spd_execute ([ndm][ld])
 *   d_out               device array of cap records (may be NULL if cap == 0)
 *   d_ws                workspace as for spd_execute
 *   use_tile_max        nonzero: d_ws still holds the tile maxima written by the
 *                       spd_execute call that produced d_snr (same plan, same
 *                       workspace, d_snr unchanged since); tiles whose maximum is
 *                       below the threshold are then skipped without being read.
 *                       0: every tile of d_snr is scanned.
 * Errors: SPD_ERR_INVALID_ARG, SPD_ERR_WORKSPACE_TOO_SMALL, SPD_ERR_CUDA.
 */
spd_status spd_candidates(const spd_plan *plan, const float *d_snr,
                          const uint16_t *d_width_idx, float threshold, int32_t peak_radius,
                          spd_candidate *d_out, int64_t cap, int64_t *d_count, void *d_ws,
                          size_t ws_bytes, int32_t use_tile_max, spd_stream_t stream);

/*
 * The synchronous overflow report of a candidate step (Sec. 4.5 candidate
 * list): waits for the stream, reads the true record count that spd_candidates,
 * spd_candidates_static, spd_search or spd_batch_candidates wrote to *d_count,
 * stores it in *total (host; may be NULL) and returns SPD_ERR_BUFFER_TOO_SMALL
 * when it exceeds cap (the list holds the first cap records in (row, start)
 * order), SPD_OK when every record was stored.  The candidate calls themselves
 * never synchronise, so that a search and its candidate step can be captured in
 * a CUDA graph; a caller that wants the error at once calls this after them.
 *   d_count  device int64 written by the candidate call (8-byte aligned)
 *   cap      the cap that call was given (>= 0)
 * Errors: SPD_ERR_INVALID_ARG, SPD_ERR_CUDA (an asynchronous error of work
 * queued on the stream, or the copy), SPD_ERR_BUFFER_TOO_SMALL.
 */
spd_status spd_candidates_status(const int64_t *d_count, int64_t cap, int64_t *total, spd_stream_t stream);

/*
 * spd_execute followed by spd_candidates(..., use_tile_max = 1) on the same
 * stream, with the same results: the candidate step reads only the tiles whose
 * maximum SNR reaches the threshold, so it adds almost no memory traffic.
 * Arguments and errors as for the two calls.
 */
spd_status spd_search(const spd_plan *plan, const void *d_x, const spd_noise *noise,
                      float *d_snr, uint16_t *d_width_idx, float threshold,
                      int32_t peak_radius, spd_candidate *d_out, int64_t cap,
                      int64_t *d_count, void *d_ws, size_t ws_bytes, spd_stream_t stream);

/*
 * spd_candidates without a workspace, for callers that cannot allocate device
 * memory when they call it: a real-time pipeline that reserves all of its
 * device memory at start-up (a later allocation can stall or fail in the
 * middle of an observation), or a plain C caller with no allocator of its own
 * for scratch space.  The paper has no counterpart; this is a deployment
 * convenience.
 *
 * Same rule, arguments, output and errors as spd_candidates with
 * use_tile_max = 0 (every tile of d_snr is scanned), minus the workspace.  Its
 * scratch is one array inside the library: per-tile counts and per-group sums
 * and offsets for at most 262,144 candidate tiles of 16,384 starts
 * (ndm * ceil(nt / 16384) tiles; 1.1 MiB, held by every device that loads the
 * library until the process exits).
 * A plan with more tiles is rejected with SPD_ERR_UNSUPPORTED before any work
 * is queued.  The call itself allocates nothing.
 *   - Each call looks up the array's device address with the device current;
 *     inside a stream capture it cannot, and uses the address found by the last
 *     call on that device outside a capture: make a first call on each device
 *     before any stream capture (and again after the device's context was
 *     destroyed and created anew, e.g. by cudaDeviceReset).
 *   - All calls on a device share the array: calls whose work overlaps on the
 *     GPU (different streams, no ordering between them) race and give wrong
 *     results.  Calls ordered on one stream are safe; nothing carries over
 *     from one call to the next.
 */
spd_status spd_candidates_static(const spd_plan *plan, const float *d_snr,
                                 const uint16_t *d_width_idx, float threshold,
                                 int32_t peak_radius, spd_candidate *d_out, int64_t cap,
                                 int64_t *d_count, spd_stream_t stream);

/*
 * Noise statistics for table-noise searches (Sec. 4.5, calculation of mean and
 * standard deviation): the per-row, per-width table that spd_execute takes
 * with spd_noise mode 1.
 *
 * For every row and every decimation level k = 0..K (2^K the smallest power of
 * two >= the plan's widest boxcar, K <= 15), the series of sums of the row's
 * complete blocks of 2^k samples gets a mean and a standard deviation
 * (population form) by point-wise outlier rejection: the first pass keeps every
 * value; each further pass keeps the values within outlier_sigma deviations of
 * the previous pass's mean, until a pass keeps as many values as the one before
 * or max_passes passes have run (outlier_sigma <= 0: one pass, no rejection).
 * Widths between powers of two are interpolated (the paper does not say how):
 * the per-sample mean mu_k / 2^k and the deviation per square-root sample
 * sigma_k / 2^(k/2) are interpolated linearly in log2(L), and
 * mu_L = L * mean, sigma_L = sqrt(L) * deviation, so white noise follows Eq.
 * whitenoise.  Levels with fewer than two values are not used: wider widths
 * extrapolate the last level with two or more values the white way; a row of
 * one sample gets sigma 0.
 *   d_x           device, [ndm][ld] samples of the plan dtype (as spd_execute)
 *   outlier_sigma rejection threshold in deviations (the paper used 2)
 *   max_passes    1..64
 *   d_mu, d_sigma device float32 [ndm][n_widths] outputs (n_widths and width
 *                 order of spd_plan_widths), 4-byte aligned
 *   d_ws          workspace of spd_workspace_size() bytes (its tile maxima are
 *                 left alone)
 * Errors: SPD_ERR_INVALID_ARG, SPD_ERR_WORKSPACE_TOO_SMALL, SPD_ERR_CUDA.  On
 * the device, when d_x is 16-byte aligned and ld x sample size is a multiple
 * of 16, the rows are read by bulk copies into shared memory (other layouts by
 * plain loads); each wait for a copy is bounded (2 s), and a row whose copy did
 * not arrive in time gets NaN in every d_mu and d_sigma entry (a search with
 * that table then has NaN SNRs in the row).
 */
spd_status spd_noise_stats(const spd_plan *plan, const void *d_x, float outlier_sigma,
                           int32_t max_passes, float *d_mu, float *d_sigma, void *d_ws,
                           size_t ws_bytes, spd_stream_t stream);

/*
 * Segment length of a BoxDIT or IGRID plan: one CTA searches `segment` starts of
 * a row (plus the widest boxcar after them, read again by the next segment).
 * Longer segments re-read less, shorter ones give more CTAs.  segment must be a
 * multiple of 16384 and of 2^top (top: the plan's last level), at most 2^24;
 * the default is the longest of 524288, 262144 and 131072 that gives at least
 * 2432 segments (ndm x segments per row).  Host only.  SPD_ERR_INVALID_ARG otherwise (and for
 * exhaustive plans).  A BoxDIT plan on the general kernel (spd_plan_create_boxdit)
 * takes tiles of 2048, 4096 or 8192 starts here instead (one CTA per tile; the
 * default is 4096 when several CTAs fit on an SM, else 2048); SPD_ERR_UNSUPPORTED
 * when a tile's shared memory would exceed 227 KB.  Such a plan above level 4
 * runs in two launches: levels 0..3 on these tiles, then levels 4.. on tiles of
 * 2048 positions of the level-4 series (32768 starts); its workspace
 * (spd_workspace_size, which depends on the tile) then also holds 14 bytes per
 * 16 samples of every row between the two.
 */
spd_status spd_plan_set_segment(spd_plan *plan, int32_t segment);

/*
 * Starts evaluated per row: only starts s < n_starts get outputs (and
 * candidates), while every sample below nt still feeds their boxcars (the rule
 * s + L <= nt of Eq. boxcar is unchanged).  For overlapping blocks of a longer
 * series, a block of n_starts + L_end - 1 samples yields exactly the outputs of
 * its n_starts starts (overlap-save).  snr / width_idx at starts >= n_starts are
 * not written; the candidate step treats n_starts as the row's end (the peak
 * test of start n_starts - 1 sees no right-hand neighbour).  1 <= n_starts <= nt;
 * the default is nt.  Host only.  SPD_ERR_INVALID_ARG otherwise.
 */
spd_status spd_plan_set_starts(spd_plan *plan, int64_t n_starts);

/*
 * Batched search of several DM ranges in one launch: ranges of different row
 * counts and lengths (e.g. the ranges of a dedispersion plan at their own time
 * decimations) searched with one grid (one BoxDIT or IGRID plan description;
 * widths, s_end and dtype are shared, in each range's own samples).  One
 * persistent kernel strides over the work list of (range, row, segment) units;
 * every launch of the library on the stream is capture-safe (CUDA graphs), but
 * the first spd_batch_execute on a device queries the device and should run
 * before a capture begins.
 *
 * Each range may name a device flag (d_ready): the units of that range wait
 * for it to become nonzero (an upstream producer writes it) before reading the
 * range.  A wait is bounded (spd_batch_set_wait_ns, default 1 s); when it runs
 * out the range is skipped (its outputs are left unwritten) and
 * spd_batch_status reports SPD_ERR_TIMEOUT.  Nothing else waits.
 *
 * Exhaustive grids and table noise are not batched (SPD_ERR_UNSUPPORTED).
 */
typedef struct spd_batch spd_batch;

typedef struct spd_range_io {
  const void *d_x;          /* [ndm][ld] samples of the grid's dtype */
  float *d_snr;             /* [ndm][ld] output, as spd_execute */
  uint16_t *d_width_idx;    /* [ndm][ld] output */
  const float *d_mu;        /* [ndm] white-noise mean of each row */
  const float *d_sigma;     /* [ndm] white-noise deviation of each row */
  const int32_t *d_ready;   /* NULL, or a device int32 flag to wait for */
} spd_range_io;

/* Creates a batch of n_ranges (1..8) ranges: row counts ndm[r], lengths nt[r],
 * row strides ld[r] (ld may be NULL: ld = nt).  grid->ndm, nt, ld are ignored.
 * Host only.  Errors as spd_plan_create. */
spd_status spd_batch_create(const spd_plan_desc *grid, const int64_t *ndm, const int64_t *nt,
                            const int64_t *ld, int32_t n_ranges, spd_batch **out);
spd_status spd_batch_destroy(spd_batch *batch);
/* Segment length of every range (rules of spd_plan_set_segment). */
spd_status spd_batch_set_segment(spd_batch *batch, int32_t segment);
/* Limit of one ready-flag wait, in nanoseconds (0..60 s). */
spd_status spd_batch_set_wait_ns(spd_batch *batch, int64_t wait_ns);
/* CTAs per SM of the persistent launch (0..64; 0, the default: as many as fit,
 * and never more than fit).  A launch-shape parameter for the autotuner; the
 * results do not depend on it. */
spd_status spd_batch_set_ctas_per_sm(spd_batch *batch, int32_t ctas_per_sm);
/* Device workspace of spd_batch_execute / spd_batch_candidates (256-byte aligned base). */
spd_status spd_batch_workspace_size(const spd_batch *batch, size_t *bytes);
/* Searches every range (io: host array of the batch's n_ranges entries), with
 * the results of spd_execute for each.  Asynchronous on stream. */
spd_status spd_batch_execute(const spd_batch *batch, const spd_range_io *io, void *d_ws,
                             size_t ws_bytes, spd_stream_t stream);
/* Waits for the stream; SPD_ERR_TIMEOUT if a ready-flag wait of the last
 * spd_batch_execute on this workspace ran out, SPD_ERR_CUDA on a CUDA error. */
spd_status spd_batch_status(const spd_batch *batch, const void *d_ws, spd_stream_t stream);
/* spd_candidates for range `range` of the last spd_batch_execute on d_ws
 * (use_tile_max: its tile maxima, as spd_candidates). */
spd_status spd_batch_candidates(const spd_batch *batch, int32_t range, const float *d_snr,
                                const uint16_t *d_width_idx, float threshold, int32_t peak_radius,
                                spd_candidate *d_out, int64_t cap, int64_t *d_count, void *d_ws,
                                size_t ws_bytes, int32_t use_tile_max, spd_stream_t stream);

/*
 * Block proposal network (no counterpart in the paper): a small 1D-conv net
 * reads x16-decimated blocks of 256 samples (4096 input samples each) and gives
 * a logit per block; blocks it flags are searched at full resolution.
 *   a1 = bf16(relu(b1 + W1 * x)), a2 = bf16(relu(b2 + W2 * a1)), h3 = b3 + W3 * a2,
 *   g[c] = max_p relu(h3[c][p]), logit = b4 + W4 . g
 * "*": correlation with kernel 9, zero padding 4; 16 channels (1 input channel
 * for layer 1); W1..W3 used as bf16, every sum in FP32 (layers 2, 3 on the
 * tensor cores).  Parameters: float32 vector of spd_net_param_count() (4817)
 * entries, W1[16][9], b1[16], W2[16][16][9], b2[16], W3[16][16][9], b3[16],
 * W4[16], b4.  Loss: binary cross-entropy of sigmoid(logit).
 */
int32_t spd_net_param_count(void);
/* Decimated series for the network: d_out[r][j] = (x[r][16j .. 16j+15] summed
 * - 16 mu_r) / (4 sigma_r), j < nt/16 (device float32 [ndm][nt/16]); d_x as
 * spd_execute for dtype; d_mu, d_sigma white-noise statistics per row. */
spd_status spd_net_decimate(const void *d_x, int32_t dtype, int64_t ndm, int64_t nt, int64_t ld,
                            const float *d_mu, const float *d_sigma, float *d_out, spd_stream_t stream);
/* Logits of n_blocks blocks (d_blocks: device float32 [n_blocks][256]). */
spd_status spd_net_forward(const float *d_params, const float *d_blocks, int64_t n_blocks,
                           float *d_logits, spd_stream_t stream);
/* Sum over the blocks of the loss gradient (d_grad_sum[4817], overwritten) and
 * of the loss (*d_loss_sum), labels d_labels[n_blocks] in {0, 1}.  The max pool
 * passes its gradient to the first maximum; roundings pass it unchanged. */
spd_status spd_net_gradient(const float *d_params, const float *d_blocks, const float *d_labels,
                            int64_t n_blocks, float *d_grad_sum, float *d_loss_sum, spd_stream_t stream);
/* spd_net_gradient with a deterministic sum: each CTA writes its partial sums
 * to its row of d_ws (device, at least spd_net_gradient_workspace_size()
 * bytes, 4-byte aligned) and a second launch adds the rows in a fixed order, so
 * equal inputs give bit-identical results (training runs are reproducible and
 * resume exactly from a checkpoint).  SPD_ERR_WORKSPACE_TOO_SMALL when ws_bytes
 * is short. */
size_t spd_net_gradient_workspace_size(void);
spd_status spd_net_gradient_ordered(const float *d_params, const float *d_blocks, const float *d_labels,
                                    int64_t n_blocks, float *d_grad_sum, float *d_loss_sum, void *d_ws,
                                    size_t ws_bytes, spd_stream_t stream);
/* One Adam step (beta 0.9, 0.999, eps 1e-8, bias-corrected; step counts from 1)
 * on the mean gradient d_grad_sum / n_blocks; d_m, d_v: moment vectors. */
spd_status spd_net_adam(float *d_params, float *d_m, float *d_v, const float *d_grad_sum,
                        int64_t n_blocks, float lr, int32_t step, spd_stream_t stream);

/* Flagged blocks: writes to d_list (device int64[cap]) the ids i < n with
 * d_logits[i] > threshold in increasing order, and their number to *d_count
 * (device int64; the full number, also when it exceeds cap, in which case only
 * the first cap ids are written). */
spd_status spd_net_select(const float *d_logits, int64_t n, float threshold, int64_t *d_list, int64_t cap,
                          int64_t *d_count, spd_stream_t stream);
/* Compact copy of blocks of a series for a restricted search: row k of d_out
 * (device [n][ld_out] of dtype; 16-byte aligned, ld_out * sample size a
 * multiple of 16) holds samples b * block - left .. b * block - left + width - 1
 * of row r of d_x, where (r, b) = (d_list[k] / bpr, d_list[k] % bpr) and
 * bpr = ceil(nt / block).  Positions outside [0, nt), the padding columns
 * width .. ld_out - 1 and rows of ids outside [0, ndm * bpr) are -inf, the value
 * the search treats as past the end of a row.  d_x as spd_execute.  F32, F16
 * and BF16 (u8 has no -inf: SPD_ERR_UNSUPPORTED). */
spd_status spd_net_gather(const void *d_x, int32_t dtype, int64_t ndm, int64_t nt, int64_t ld,
                          const int64_t *d_list, int64_t n, int32_t block, int32_t left, int32_t width,
                          void *d_out, int64_t ld_out, spd_stream_t stream);

/*
 * Proposal search: the network above flags 4096-sample blocks, and only the
 * flagged blocks are searched at full resolution with the plan grid; all of it
 * runs on the device, records come back in the series' own (row, start).
 *
 * spd_proposal_create: grid is a plan description of the series (algo, dtype,
 * s_end, boxdit_lmax, igrid_*, ndm, nt, ld) with nt a multiple of 4096 and
 * dtype F32, F16 or BF16 (U8: SPD_ERR_UNSUPPORTED); peak_radius (0..64) is the
 * candidate rule's R; max_blocks (>= 1; clamped to ndm * nt / 4096) bounds the
 * flagged blocks one call can search and sizes the workspace.  Each flagged
 * block is searched in a compact row holding L samples before it (L the
 * smallest multiple of the grid's largest start separation >= max(R, 1)), the
 * block, and R + the widest boxcar after it (-inf outside the series), so every
 * start of the block and of its peak-test neighbours gets the outputs of a
 * search of the whole row.  The grid's
 * start separations must divide 4096 (else SPD_ERR_UNSUPPORTED).  Host only.
 */
typedef struct spd_proposal spd_proposal;
spd_status spd_proposal_create(const spd_plan_desc *grid, int32_t peak_radius, int64_t max_blocks,
                               spd_proposal **out);
spd_status spd_proposal_destroy(spd_proposal *prop);
/* Device workspace of spd_propose_search in bytes (256-byte aligned base). */
spd_status spd_proposal_workspace_size(const spd_proposal *prop, size_t *bytes);
/* The grid's widths and separations (as spd_plan_widths); the width indices of
 * the records and the width order of a noise table refer to it. */
spd_status spd_proposal_widths(const spd_proposal *prop, int32_t *widths, int32_t *seps, int32_t cap,
                               int32_t *n);
/*
 * One proposal search of the series d_x ([ndm][ld] of the grid's dtype):
 *   1. decimated blocks (spd_net_decimate with the width-1 statistics of
 *      `noise`), logits (spd_net_forward with d_params), and the ids of the
 *      blocks whose logit > logit_threshold (spd_net_select);
 *   2. the number of flagged blocks is read back (the stream is synchronised
 *      once) and written to *n_blocks (host, may be NULL); more than max_blocks:
 *      SPD_ERR_BUFFER_TOO_SMALL, nothing searched; none: *d_count = 0;
 *   3. the flagged blocks and their rows' statistics are gathered, searched
 *      (spd_execute on the compact rows) and their candidates selected with
 *      threshold and the proposal's peak radius (spd_candidates rule), only
 *      starts inside a block counting; records carry the series' row and start,
 *      in (row, start) order, with the grid's width index and width.
 * noise: mode 0, mu/sigma [ndm]; mode 1, [ndm][n_widths] of the grid (device).
 * d_out, cap, d_count as spd_candidates (first cap records, true count; see
 * spd_candidates_status).  Asynchronous after step 2; errors as spd_execute.
 */
spd_status spd_propose_search(const spd_proposal *prop, const float *d_params, const void *d_x,
                              const spd_noise *noise, float logit_threshold, float threshold,
                              spd_candidate *d_out, int64_t cap, int64_t *d_count, int64_t *n_blocks,
                              void *d_ws, size_t ws_bytes, spd_stream_t stream);
/*
 * Step 3 of spd_propose_search alone, for blocks the caller chose: d_ids
 * (device int64[n_ids], increasing) are block ids r * (nt / 4096) + b of the
 * series.  n_ids above the proposal's max_blocks: SPD_ERR_BUFFER_TOO_SMALL;
 * 0: *d_count = 0.  An id outside [0, ndm * nt / 4096) is searched as a block
 * of -inf samples (no records).  Asynchronous; other arguments and errors as
 * spd_propose_search.
 */
spd_status spd_search_blocks(const spd_proposal *prop, const void *d_x, const spd_noise *noise,
                             const int64_t *d_ids, int64_t n_ids, float threshold, spd_candidate *d_out,
                             int64_t cap, int64_t *d_count, void *d_ws, size_t ws_bytes, spd_stream_t stream);

/*
 * Wait for the stream and report any asynchronous CUDA error of work queued
 * on it (SPD_ERR_CUDA), else SPD_OK.
 */
spd_status spd_sync_status(const spd_plan *plan, spd_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SPD_H */
