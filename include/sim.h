/*
 * sim.h -- C ABI of the GB300 charge-readout simulation of a pixelated LArTPC
 * (arXiv:2212.09807, "Highly-parallelized simulation of a pixelated LArTPC on
 * a GPU", Sec. 3).
 *
 * Conventions shared by every entry point:
 *  - Pointers are DEVICE pointers unless marked (host).  The caller owns every
 *    buffer; the library allocates nothing on the device.
 *  - Every call is asynchronous on the caller's CUDA stream (`stream` is a
 *    cudaStream_t passed as void*; NULL = the legacy default stream).  No call
 *    synchronises the host.
 *  - Host-side argument checks run before any launch; a failed check returns
 *    SIM_ERR_INVALID_ARG and enqueues nothing.
 *  - Counts that only the device knows (pairs, active pixels, hits) are written
 *    to device int64 words.  When a count exceeds the caller's capacity the
 *    kernels skip the writes that would overflow, store the required size and
 *    set a bit in the status word (see SIM_STATUS_*); the caller reads the
 *    counts after synchronising, grows its buffers and calls again.
 *  - Units: cm, us, MeV, electrons.  Pixel ids are global int32:
 *      anode = (my * n_mod_x + mx) * n_tpc + tpc,
 *      pixel = anode * (npx_x * npx_y) + iy * npx_x + ix,
 *    npx_x = tiles_x * px_per_tile, npx_y = tiles_y * px_per_tile.
 *  - Results depend only on (config, segments, event_id, seed), not on thread
 *    order or batch composition (the paper's requirement that a result must
 *    not depend on the order of execution of the threads, Sec. 2).  The
 *    tensor-core current forms (sim_config.precision 1, 2) are bitwise
 *    reproducible call by call; across batch compositions or pixel slices
 *    their currents agree to their accumulation rounding (~1e-7).
 */
#ifndef LARPIX_GB300_SIM_H
#define LARPIX_GB300_SIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define SIM_OK 0
#define SIM_ERR_INVALID_ARG (-1) /* null pointer, negative size, bad config: nothing enqueued */
#define SIM_ERR_CAPACITY (-2)    /* a host-known size exceeds a buffer or the workspace */
#define SIM_ERR_CUDA (-3)        /* a CUDA launch or copy failed; see sim_last_cuda_error() */
#define SIM_ERR_TIMEOUT (-4)     /* reserved: a bounded device-side wait gave up */

/* Bits of the device status word (workspace counts block, index 3). */
#define SIM_STATUS_PAIR_OVERFLOW 1
#define SIM_STATUS_PIXEL_OVERFLOW 2
#define SIM_STATUS_HIT_OVERFLOW 4
#define SIM_STATUS_TICK_RANGE 8
#define SIM_STATUS_TIMEOUT 16     /* a bounded device-side wait gave up (tensor-core form) */

/* Simulation parameters (host struct, copied at each call).  Floating-point
 * fields are FP32.  Citations: recombination Sec. 3.1 Eq. (birks)/(box);
 * drift Sec. 3.2; sampling Sec. 3.3.2; front end Sec. 3.4; geometry Sec. 6. */
typedef struct sim_config {
    /* geometry: modules tile x-y; TPC 0 anode at z=0, cathode at z=drift_len,
     * TPC 1 anode at z=2*drift_len */
    int32_t n_mod_x, n_mod_y, n_tpc, tiles_x, tiles_y, px_per_tile;
    float pitch_cm, drift_len_cm;
    /* recombination: 0 = Birks, 1 = modified Box */
    int32_t recomb_model;
    float birks_Ab, birks_kb, box_alpha, box_beta, efield_kV_cm, lar_density_g_cm3, w_ion_MeV;
    /* drift */
    float vdrift_cm_us, lifetime_us, diff_long_cm2_s, diff_tran_cm2_s;
    /* sampling of Eq. (current): point spacing, perturbations per point, clip (sigmas) */
    float sample_step_cm;
    int32_t mc_per_sample;
    float diff_clip_sigma;
    /* readout window: tick length, number of ticks, start time */
    float tick_us;
    int32_t n_ticks;
    float t_window0_us;
    /* front end */
    float thr_e, sigma_reset_e, sigma_disc_e, sigma_unc_e, gain_e_per_mV, adc_lsb_mV;
    int32_t hold_ticks, min_adc_interval_ticks, periodic_reset_ticks, adc_bits;
    /* counter-based RNG seed (Philox4x32-10 key = seed ^ event_id) */
    uint64_t seed;
    /* arithmetic form of the induced-current step (sim_induced_current):
     * 0 = FP32 form on the CUDA cores (charge binned per table node); 1 =
     * tensor-core contraction with BF16 operands, 2 = with FP16 operands (FP32
     * accumulation in both); 3 = FP32 term-by-term gather (each point record's
     * bilinear and linear table reads summed directly: slower, kept as an
     * independent FP32 evaluation) */
    int32_t precision;
    /* running CSA charge of the front end (sim_electronics): 0 = FP32,
     * 1 = FP64 (for long windows, where FP32 sums drift); decisions compare
     * FP32 roundings either way */
    int32_t fp64_charge;
    /* optional device bitmask of disabled channels (bit p % 32 of word p / 32
     * set: detector pixel id p is disabled; NULL: none).  A disabled pixel's
     * current is computed but its front end produces no hits; in a batch the
     * mask applies to every event slot. */
    const uint32_t *disabled_pixels;
    /* 0: lifetime and diffusion evaluated once per segment, at its midpoint
     * (Sec. 3.2); 1: at each point's own drift distance: a point carries
     * Q_a/(N M) exp(-(t_point - t_drift)/tau) and diffuses with
     * sqrt(2 D t_point); sim_quench_drift then reports sigma_T/L of the
     * segment's farther end (they bound every point's, and size the map) */
    int32_t per_point_drift;
    /* table lookup: 0 = bilinear in the folded offset and linear in the
     * arrival tick; 1 = nearest node and nearest tick (halves round up) */
    int32_t nearest_lut;
    /* scheduling shapes of the induced-current step (results do not depend on
     * them beyond the accumulation rounding; 0 = default): tensor-core forms:
     * target work units per SM of the work plan (1..16, default 2) and records
     * per CTA chunk (a power of two, 4096..1048576; default 1048576 for calls
     * sized for at least 131072 active pixels, else 262144; the workspace holds
     * two record buffers of 32 bytes per record and CTA); FP32 form: resident
     * CTAs per SM (1..4, default 4; results bitwise the same for every value)
     * and, from tc_record_chunk, the records per chunk of a pixel (at most and
     * by default 65520).  paper_2212_09807_gb300/tune.py picks them by timing a
     * sample. */
    int32_t tc_units_per_sm, tc_record_chunk, direct_ctas_per_sm;
    /* polls of a bounded device-side wait of the tensor-core forms before it
     * gives up (0 = default 2^22, about two seconds; 1 .. 2^30).  A wait that
     * gives up sets SIM_STATUS_TIMEOUT and the kernel winds down: its results
     * are then invalid, and it still waits (with the default bound) for the
     * MMAs and copies it has issued before it returns.  Lowering it makes the
     * waits of a normal call give up: this is how the timeout path is tested. */
    int32_t wait_spin_limit;
} sim_config;

/* Energy-deposit segments S_i = (r_s, r_e, E) (Sec. 2), as structure-of-arrays
 * FP32 device columns of length n: start (x0,y0,z0,t0), end (x1,y1,z1,t1),
 * deposited energy dE.
 *  - n_events == 0: one event with id event_id; segment index i keys the
 *    diffusion random numbers together with event_id.
 *  - n_events >= 1 (a batch): event slot e owns segments
 *    [event_offsets[e], event_offsets[e+1]) and has id event_ids[e]
 *    (device arrays of n_events + 1 and n_events entries, offsets increasing,
 *    event_offsets[0] = 0, event_offsets[n_events] = n); its random numbers use
 *    the event-local segment index, so every event's results are identical alone
 *    and in a batch.  Pixel ids then refer to a virtual detector with one copy of
 *    the geometry per slot: virtual id = slot * n_detector_pixels + pixel id. */
typedef struct sim_segments {
    const float *x0, *y0, *z0, *t0, *x1, *y1, *z1, *t1, *dE;
    int64_t n;
    uint64_t event_id;
    const int64_t *event_offsets;
    const uint64_t *event_ids;
    int64_t n_events;
} sim_segments;

/* Field-response table I_pixel[x, y, t] (Sec. 3.3.1): FP32 device array
 * [nb][nb][ld], series of nt ticks (electrons per tick for one electron; row
 * nt-1 is the last tick before arrival) at folded offsets
 * (b + 1/2) * pitch / bins_per_pitch, b = 0..nb-1.  ld >= nt, ld % 4 == 0,
 * the row tail [nt, ld) is ignored. */
typedef struct sim_response {
    const float *lut;
    int32_t nb, nt, ld, bins_per_pitch;
} sim_response;

/* Per-segment results of sim_quench_drift (device arrays of length n):
 * Q_a (electrons at the anode), t_drift (us), sigma_T, sigma_L (cm), anode
 * (-1 = inactive segment), n_samples (points N along the segment), and
 * `anchors`: SIM_ANCHOR_BYTES per segment, 16-byte aligned, an opaque
 * sampling record read by sim_pixel_map and sim_induced_current. */
#define SIM_ANCHOR_BYTES 64
typedef struct sim_drifted {
    float *Qa, *t_drift, *sigma_T, *sigma_L;
    int32_t *anode, *n_samples;
    void *anchors;
} sim_drifted;

/* Hit list written by sim_electronics / sim_event, ordered by active-pixel
 * index then tick: pixel id, threshold-crossing tick, ADC tick, 8-bit ADC
 * code and the digitised CSA charge (electrons).  n_out (device int64)
 * receives the number of hits (which may exceed capacity: see status). */
typedef struct sim_hits {
    int32_t *pixel, *t_cross, *t_adc;
    uint8_t *adc;
    float *q;
    int64_t capacity;
    int64_t *n_out;
} sim_hits;

/* Human-readable text of a return code (static string). */
const char *sim_strerror(int code);

/* The cudaError_t of the last SIM_ERR_CUDA return of this host thread. */
int sim_last_cuda_error(void);

/* Sizes of the ABI structs as compiled (for binding checks): writes
 * sizeof(sim_config), sizeof(sim_segments), sizeof(sim_response),
 * sizeof(sim_drifted), sizeof(sim_hits) to sizes[0..4] (host). */
void sim_abi_sizes(int64_t sizes[5]);

/* Workspace bytes sim_event needs for batches of up to max_events events
 * (0 or 1 for a single event), max_segments segments, max_pairs (segment,
 * pixel) pairs and max_pixels active pixels, on the current device; the same
 * size serves sim_pixel_map, sim_induced_current and sim_electronics, which use
 * only the scratch region after the counts block.  Writes *bytes (host).  The
 * first 256 bytes of any workspace hold the counts block: int64 [0] pairs,
 * [1] active pixels, [2] hits, [3] status bits (SIM_STATUS_*). */
int sim_workspace_size(const sim_config *cfg, int64_t max_events, int64_t max_segments,
                       int64_t max_pairs, int64_t max_pixels, size_t *bytes);

/* Device address of the counts block inside a workspace. */
const int64_t *sim_workspace_counts(const void *ws);

/* Steps 1-2 (Sec. 3.1 Eq. (birks)/(box); Sec. 3.2 Eq. (drift), Eq. (lifetime),
 * sigma = sqrt(2 D t_drift)): one pass over the segments.
 *   R   = A_b / (1 + k_b/eps dE/dx)            (Birks, default)
 *       = ln(alpha + xi) / xi, xi = beta/eps dE/dx  (modified Box)
 *   Q_a = R (dE / W_ion) exp(-t_drift / tau), t_drift = |z_mid - z_anode| / v_drift
 * Segments whose midpoint is outside every drift volume, or shorter than
 * 1e-6 cm, get anode = -1 and Q_a = 0. */
int sim_quench_drift(const sim_config *cfg, const sim_segments *seg, const sim_drifted *out,
                     void *stream);

/* Step 3 (Sec. 3.3.2, pixels a segment can induce on).  Pixel p of the
 * segment's anode is mapped iff the segment's x-y projection comes within
 * Chebyshev distance (nb + 1/2) pitch/bins_per_pitch + clip * sigma_T of its
 * centre (nb and bins_per_pitch from `resp`; its table is not read).  Outputs:
 *   seg_pix_off [n+1], seg_pix_ids [pair_cap]   segment -> pixel ids (CSR)
 *   active_pixels [pix_cap]                      mapped pixel ids, increasing
 *   pix_seg_off [pix_cap+1], pix_seg_ids [pair_cap]  pixel -> segments (CSR,
 *                                                segment indices increasing)
 * Counts go to the workspace counts block ([0] pairs, [1] pixels, [3] status);
 * on overflow the required sizes are stored and the CSR fill is skipped.
 * Workspace: sim_workspace_size(cfg, n_events, n, pair_cap, pix_cap). */
int sim_pixel_map(const sim_config *cfg, const sim_segments *seg, const sim_drifted *dr,
                  const sim_response *resp, int32_t *seg_pix_off, int32_t *seg_pix_ids, int64_t pair_cap,
                  int32_t *active_pixels, int32_t *pix_seg_off, int32_t *pix_seg_ids,
                  int64_t pix_cap, void *ws, size_t ws_bytes, void *stream);

/* Step 4 (Sec. 3.3.2, charge density rho and Eq. (current)):
 *   I[p, k] = sum over segments s mapped to p, points mu < N_s, perturbations
 *             nu < M of q_s * Rt(x - x_p, y - y_p, k - a),  q_s = Q_a/(N_s M),
 * the table read bilinearly at the folded transverse offset and linearly at
 * the fractional arrival tick a.  current: FP32 [pix_cap][n_ticks]; rows
 * [0, counts[1]) are written.  counts: device int64[6] counts block as
 * written by sim_pixel_map ([1] = active pixels, [3] = status); nothing is
 * computed when the status word is nonzero or counts[1] > pix_cap.
 * Every form regroups the terms as I[p, k] = sum over table nodes n and
 * arrival ticks a of Q[p, n, a] R[n, k - a + L - 1] (Q: charge deposited on
 * node n at tick a by the linear weights, accumulated in fixed point with
 * integer atomics); cfg->precision selects the arithmetic of the sum:
 * 0 FP32 on the CUDA cores (Q at a power-of-two scale per chunk of a pixel's
 * points, ~1e-9 of its charge; partial sums added into compensated totals);
 * 3 FP32 without the regrouping: each point record's terms summed per tick
 * (the table rows of its bin staged in shared memory; records of a chunk in
 * point order, bins increasing; chunk sums added into compensated totals);
 * 1 (BF16) and 2 (FP16) contract Q with the Toeplitz blocks of each table row
 * on the tensor cores (Q in fixed point 2^-12 e-, then rounded to the operand
 * type, as is R; FP16 Q cells saturate at 262016 e-).  Results are bitwise
 * reproducible for a given call, and with precision 0 or 3 a pixel's current
 * does not depend on the other pixels of the call; counts[4] receives the number
 * of tensor-core MMA instructions (M = 128, N = 32, K = 16) of the call and
 * counts[5] the number of nonzero charge cells Q[p, n, a] it summed, and
 * SIM_STATUS_TIMEOUT is set if a bounded device-side wait gave up.
 * Workspace (scratch from byte 256 on): sim_workspace_size(cfg, 0, 0, 0,
 * pix_cap) bytes, sized for the current device (per-CTA record buffers, up to
 * ~2.5 GB for precision 0 and 0.24 GB for 3 on 152 SMs; with precision 1/2
 * also the phase tables).  Table limits: nb * nb <= 2048, nt <= 2048. */
int sim_induced_current(const sim_config *cfg, const sim_segments *seg, const sim_drifted *dr,
                        const sim_response *resp, const int32_t *active_pixels,
                        const int32_t *pix_seg_off, const int32_t *pix_seg_ids,
                        const int64_t *counts, int64_t pix_cap, float *current, void *ws,
                        size_t ws_bytes, void *stream);

/* Step 4 on a slice of the active pixels: as sim_induced_current, but only the
 * rows of active pixels [pix_begin, min(counts[1], pix_end)) are computed and
 * written (rows are indexed by active-pixel index, as in the full call).  Each
 * pixel's current is the same as the full call's: the FP32 form bit for bit,
 * the tensor-core form up to its accumulation rounding (its pixel groups are
 * formed within the slice).  Lets a caller cut a large event's current step
 * into shorter launches (other streams' work interleaves between them).
 * 0 <= pix_begin <= pix_end; an empty slice is a no-op. */
int sim_induced_current_range(const sim_config *cfg, const sim_segments *seg, const sim_drifted *dr,
                              const sim_response *resp, const int32_t *active_pixels,
                              const int32_t *pix_seg_off, const int32_t *pix_seg_ids,
                              const int64_t *counts, int64_t pix_begin, int64_t pix_end,
                              int64_t pix_cap, float *current, void *ws, size_t ws_bytes,
                              void *stream);

/* Step 5 (Sec. 3.4): per active pixel, tick by tick, charge integration,
 * discriminator with uncorrelated and threshold noise, hold, 8-bit ADC and
 * reset with pedestal noise (Philox counters keyed by pixel id and tick).
 * Reads counts[1] (active pixels) and counts[3] (status; nothing is done when
 * nonzero); writes the hit list `out`, *out->n_out and counts[2] (hits).
 * `events` supplies the event ids only (event_id, or event_ids/n_events of a
 * batch; its segment columns are not read).
 * Workspace (scratch, from byte 256 on): sim_workspace_size(cfg, 0, 0, 0, pix_cap). */
int sim_electronics(const sim_config *cfg, const sim_segments *events, const int32_t *active_pixels,
                    const float *current, int64_t *counts, int64_t pix_cap,
                    const sim_hits *out, void *ws, size_t ws_bytes, void *stream);

/* Steps 1-5 for one event or a batch of events (see sim_segments), enqueued
 * on one stream with no host synchronisation; every intermediate lives in the
 * workspace, sized by sim_workspace_size(cfg, seg->n_events, seg->n, max_pairs,
 * max_pixels). */
int sim_event(const sim_config *cfg, const sim_segments *seg, const sim_response *resp,
              int64_t max_pairs, int64_t max_pixels, const sim_hits *out, void *ws,
              size_t ws_bytes, void *stream);

/* Allocation-free pixel map.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc when they map an event, such
 * as services that fix their device-memory budget at start-up and must not
 * allocate in their event loop, or code embedded in a framework whose
 * allocator owns all device memory.  Same inputs, outputs and results as
 * sim_pixel_map, with the counts block (device int64[4], written as by
 * sim_pixel_map) passed explicitly; its scratch lives in a file-scope device
 * array of SIM_NOALLOC_SCRATCH_BYTES that every device loading this library
 * holds until the process exits.  The call allocates nothing.
 *  - Returns SIM_ERR_CAPACITY, with nothing enqueued, when the event needs more
 *    scratch than that: 2 x 4 x (total pixels + 1) bytes plus the scan's tile
 *    sums, i.e. detectors of up to about two million pixels.
 *  - The first call on a device looks up the array's device address (a host
 *    call, cudaGetSymbolAddress); make that first call before any stream
 *    capture.
 *  - All calls share the array: calls whose work overlaps on the GPU race and
 *    must be ordered by the caller (one stream, or events between streams).
 *  - The looked-up address is cached per device for the life of the process;
 *    it is invalid after cudaDeviceReset on that device, so a process that
 *    resets a device must not call this entry point on it afterwards. */
#define SIM_NOALLOC_SCRATCH_BYTES (16u << 20)
int sim_pixel_map_noalloc(const sim_config *cfg, const sim_segments *seg, const sim_drifted *dr,
                          const sim_response *resp, int32_t *seg_pix_off, int32_t *seg_pix_ids,
                          int64_t pair_cap, int32_t *active_pixels, int32_t *pix_seg_off,
                          int32_t *pix_seg_ids, int64_t pix_cap, int64_t *counts, void *stream);

/* Device addresses of sim_event's intermediates inside its workspace (for
 * inspection after the stream has run): per-segment results, both CSR maps,
 * the active-pixel list, the induced current [max_pixels][n_ticks] and the
 * counts block. */
typedef struct sim_event_view {
    sim_drifted dr;
    int32_t *seg_pix_off, *seg_pix_ids, *active_pixels, *pix_seg_off, *pix_seg_ids;
    float *current;
    int64_t *counts;
} sim_event_view;

int sim_event_view_of(const sim_config *cfg, int64_t max_events, int64_t n_segments,
                      int64_t max_pairs, int64_t max_pixels, void *ws, size_t ws_bytes,
                      sim_event_view *view);

/* Measurement support (no counterpart in the paper): enqueues a kernel of
 * `blocks` CTAs of 256 threads that issues only independent FP32 fused
 * multiply-adds, iters x 128 per thread, and writes the flops it performs to
 * *flops (host).  Timed with events on `stream`, it gives the device's FP32
 * FMA rate, the bound of the FP32 form of sim_induced_current.  sink:
 * device FP32 [blocks * 256] (never written in practice; it keeps the
 * arithmetic live).  1 <= blocks <= 2^20, iters >= 1. */
int sim_probe_fma(int64_t blocks, int32_t iters, float *sink, double *flops, void *stream);

/* ---------------------------------------------- after the front end ---- */

/* Running sums of the response table rows, for sim_hit_truth, stored as quads
 * of the four rows a bilinear read combines: cum is FP32 [nb][nb][ld][4] (16 *
 * nb * nb * ld bytes, 16-byte aligned) and cum[bx][by][j][c] = sum over
 * j' <= j of resp->lut[bx + dx][by + dy][j'], (dx, dy) = (c & 1, c >> 1), for
 * j < nt (accumulated in FP64, rounded to FP32; 0 for rows beyond the table;
 * positions [nt, ld) are not written).  Compute it once per table. */
int sim_response_cumulative(const sim_response *resp, float *cum, void *stream);

/* Per-hit charge truth written by sim_hit_truth (device arrays; the caller
 * owns them): for hit h (the hit list's order), entries h*k .. h*k+k-1 of
 * `segment` and `q` list the segments that induced the largest |charge| on
 * the hit's pixel during the ticks the hit digitises, in decreasing |charge|
 * (ties: lower segment index first), as indices into the call's segment
 * arrays and electrons; unused entries hold -1 and 0.  q_signal[h] is the
 * charge of all the pixel's segments in those ticks (the hit's signal,
 * without front-end noise and pedestal).  tick_first (optional, NULL = not
 * written) receives the first tick of each hit's interval. */
#define SIM_TRUTH_MAX_K 16
typedef struct sim_truth {
    int32_t k;                 /* entries per hit, 1 .. SIM_TRUTH_MAX_K */
    int32_t *segment;          /* [capacity * k] */
    float *q;                  /* [capacity * k] */
    float *q_signal;           /* [capacity] */
    int32_t *tick_first;       /* [capacity] or NULL */
    int64_t capacity;          /* hits */
} sim_truth;

/* Charge truth of every hit (Sec. 3.4 with the truth scheme of Sec. 4.4
 * applied to the charge readout).  A hit digitises the current of ticks
 * [k0, k1]: k1 is its ADC tick; k0 the tick after the previous hit's ADC tick
 * on the same pixel (0 for the first), or the latest periodic reset tick
 * r = j * periodic_reset_ticks with k0 < r <= its crossing tick.  The charge
 * segment s put there is sum_{k=k0}^{k1} of the terms of Eq. (current) that
 * come from s, the same terms sim_induced_current sums (for any precision
 * setting they are evaluated in FP32 from the table's running sums `cum`,
 * sim_response_cumulative), summed exactly in fixed point (2^-16 e-) per
 * (hit, segment).  Inputs: the segment, drift and map outputs of the event (or
 * batch) and the hit list of sim_electronics / sim_event (pixel ids, crossing
 * and ADC ticks, ordered by pixel then tick; *hits->n_out hits, at most
 * min(hits->capacity, out->capacity) processed).
 * Workspace: sim_hit_truth_workspace_size(min(hits->capacity, out->capacity),
 * max_cells) bytes; its first 256 bytes hold int64 counts: [0] cells needed
 * (sum over the hits' pixels of hits x mapped segments), [1] runs (hit pixels),
 * [2] work units, [3] status (bit 1: more than max_cells cells; nothing was
 * computed and q_signal is 0).  Nothing is computed either when counts[3] of
 * the map reports an overflow.  Results are bitwise reproducible. */
int sim_hit_truth_workspace_size(int64_t max_hits, int64_t max_cells, size_t *bytes);
int sim_hit_truth(const sim_config *cfg, const sim_segments *seg, const sim_drifted *dr,
                  const sim_response *resp, const float *cum, const int32_t *active_pixels,
                  const int32_t *pix_seg_off, const int32_t *pix_seg_ids, const int64_t *counts,
                  int64_t pix_cap, const sim_hits *hits, const sim_truth *out, int64_t max_cells,
                  void *ws, size_t ws_bytes, void *stream);

/* Hits -> 3-D points (Sec. 6): x, y = centre of the hit's pixel (global cm),
 * z from the crossing tick by the inverse of Eq. (drift): the tick starts at
 * t = t_window0 + t_cross * tick, and z = z_anode + v_d (t - t_event) for an
 * anode at z = 0, z_anode - v_d (t - t_event) for the anode at 2 drift_len.
 * t_event: device FP32 array with the event time of each event slot of the
 * hits' (virtual) pixel ids, or NULL (all events at t = 0).  Writes x, y, z
 * [hits->capacity] for the first min(*hits->n_out, capacity) hits, evaluated
 * in FP64 and rounded to FP32. */
int sim_hit_points(const sim_config *cfg, const sim_hits *hits, const float *t_event, float *x, float *y,
                   float *z, void *stream);

/* dQ/dx along a known straight track (Sec. 6, the charge per unit length of a
 * track's hits, in pieces of length piece_cm): point i (x, y, z: device FP32
 * arrays of `capacity`, *n_points of them used, n_points a device int64) at
 * arc length s = (p - origin) . direction (direction: unit vector) and
 * distance d from the line belongs to piece floor(s / piece_cm) when
 * 0 <= s < n_pieces piece_cm and d <= r_max_cm; dq[b] (device FP64) receives
 * the sum of charges q (device FP32) of piece b and count[b] (device int32)
 * its points.  Decisions are IEEE FP64 evaluations of these expressions;
 * charges are summed exactly in fixed point (2^-16 e-).  origin, direction:
 * host arrays of 3. */
int sim_track_dqdx(const float *x, const float *y, const float *z, const float *q, const int64_t *n_points,
                   int64_t capacity, const double *origin, const double *direction, double piece_cm,
                   int32_t n_pieces, double r_max_cm, double *dq, int32_t *count, void *stream);

/* ------------------------------------------------------------ light ---- */
/* Light path of Sec. 4 on the same segments: photon yield and photoelectrons
 * per photosensor (Sec. 4.1), photocurrent from the arrival-time table
 * (Sec. 4.2), the truncated scintillation convolution, counting fluctuations,
 * and the electronics response with noise, sampling and ADC (Sec. 4.3).
 * Photosensor ids: det = anode * n_det + k (anode as in sim_drifted.anode),
 * n_det photosensors per TPC; a call covers all n_anodes * n_det of them
 * (n_anodes = n_mod_x * n_mod_y * n_tpc; single events only).  Tables describe
 * one TPC in local coordinates: x, y from the module corner, z = distance from
 * the anode, cubic voxels of vox_cm from that corner. */
typedef struct sim_light_config {
    const float *vis;          /* [nvx][nvy][nvz][n_det] visibility V_i */
    const float *tdist;        /* [nvx][nvy][nvz][n_det][nt] arrival-time fractions per tick (rows sum to 1) */
    const float *eff;          /* [n_det] detection efficiency eps_i */
    const float *gain;         /* [n_det] G_i, ADC per photoelectron */
    const float *resp;         /* [n_resp] impulse response, unit sum, one tick per bin */
    const float *noise_amp;    /* [noise_block / 2 + 1] amplitudes A_k of the noise spectrum (ADC) */
    int32_t nvx, nvy, nvz, n_det, nt, n_resp, noise_block, adc_bits;
    float vox_cm, w_ph_MeV;    /* voxel edge; energy per photon at zero field */
    float tick_us, t_start_us; /* light tick and window start */
    int32_t n_ticks, pad0;     /* window length */
    float fast_frac, tau_fast_us, tau_slow_us, trunc_taus, poisson_max_mean;
    float sample_us, pedestal_adc;
} sim_light_config;

/* Number of digitiser samples of the window: floor((n_ticks - 1) tick_us /
 * sample_us) + 1 (ratio formed in FP64 from the FP32 fields). */
int sim_light_n_samples(const sim_light_config *lc, int64_t *n_samples);

/* Sec. 4.1 per segment (thread per segment): photons N_gamma = dE / W_ph - Q_R
 * (Q_R = Q_a e^(t_drift / lifetime), the quenched ionisation of Sec. 3.1;
 * floored at 0), photoelectrons npe[i][k] = eff[k] vis[voxel][k] N_gamma at
 * the voxel of the midpoint, and tick[i] = floor((t_mid - t_start) / tick)
 * of the midpoint time; voxel and tick are decided with IEEE FP32 operations
 * in that order (voxel indices clamped to the table).  Inactive segments
 * (anode < 0): npe 0, vox -1.  npe: FP32 [n][n_det]; tick, vox: int32 [n]. */
int sim_light_yield(const sim_config *cfg, const sim_light_config *lc, const sim_segments *seg,
                    const sim_drifted *dr, float *npe, int32_t *tick, int32_t *vox, void *stream);

/* Sec. 4.2, Eq. (photocurrent) with table and simulation ticks equal:
 * pe[det][t] = sum over the segments j of det's anode of
 * tdist[vox_j][k][t - tick_j] npe[j][k] (0 <= t - tick_j < nt), as 64-bit
 * fixed point of 2^-16 photoelectrons (each term rounded once; the sum is
 * exact, hence independent of order).  pe_fix: int64 [n_anodes * n_det][n_ticks],
 * overwritten.  Limits: n_det <= 32, nt <= 256. */
int sim_light_photocurrent(const sim_config *cfg, const sim_light_config *lc, const sim_segments *seg,
                           const sim_drifted *dr, const float *npe, const int32_t *tick, const int32_t *vox,
                           int64_t *pe_fix, void *stream);

/* Sec. 4.2, the truncated scintillation convolution
 * S[t] = sum_{u=0}^{min(t, N)} pe[t - u] f_scint(u tick),
 * f_scint(t) = f_p / tau_p e^(-t / tau_p) + (1 - f_p) / tau_s e^(-t / tau_s),
 * N = floor(trunc_taus tau_s / tick + 1/2), computed as the exactly
 * equivalent pair of first-order recurrences (one per component) with the
 * truncated tail subtracted.  scint: FP32 [n_anodes * n_det][n_ticks]
 * (photoelectrons per us). */
int sim_light_scintillation(const sim_config *cfg, const sim_light_config *lc, const int64_t *pe_fix,
                            float *scint, void *stream);

/* Sec. 4.2, counting fluctuations per tick: lambda = S[t] tick; lambda <=
 * poisson_max_mean: the smallest n with u <= F(n) (Poisson CDF accumulated in
 * FP64, at most 1000 terms), u from Philox block (det, t, 5, 0); above: a
 * normal lambda + sqrt(lambda) z (Philox block (det, t, 6, 0)), floored at 0.
 * Key seed ^ event_id.  pe_obs: FP32 [n_anodes * n_det][n_ticks]. */
int sim_light_fluctuate(const sim_config *cfg, const sim_light_config *lc, uint64_t event_id, const float *scint,
                        float *pe_obs, void *stream);

/* Sec. 4.3: V[t] = noise(t) + gain[k] sum_{u < n_resp} pe_obs[t - u] resp[u],
 * noise on blocks of noise_block ticks (b = t / N, tau = t - b N):
 * sum_{k <= N/2} A_k cos(2 pi k tau / N + phi_k), phi_k = 2 pi u of Philox
 * block (det, b, 7, k) (an inverse FFT per block); then sample m at
 * p = m sample_us / tick_us, read linearly between ticks floor(p) and
 * floor(p) + 1, code = clamp(floor(v + pedestal + 1/2), 0, 2^adc_bits - 1).
 * v: FP32 [n_anodes * n_det][n_ticks], overwritten (the analog waveform);
 * wave: uint16 [n_anodes * n_det][n_samples].  noise_block: a power of two,
 * 64 .. 4096; n_resp <= 2048. */
int sim_light_electronics(const sim_config *cfg, const sim_light_config *lc, uint64_t event_id,
                          const float *pe_obs, float *v, uint16_t *wave, void *stream);

/* Sec. 4.4, the default light truth: for each segment and photosensor k of
 * its TPC, the photoelectrons npe[i][k] of sim_light_yield and their mean
 * arrival time (us) on the simulation's tick grid, before the scintillation
 * delay: t_arrival[i][k] = t_start + (tick[i] + sum_u (u + 1/2)
 * tdist[vox[i]][k][u]) tick (FP64, rounded to FP32; 0 for vox < 0).
 * tick, vox: from sim_light_yield; t_arrival: FP32 [n_segments][n_det]. */
int sim_light_truth(const sim_config *cfg, const sim_light_config *lc, int64_t n_segments, const int32_t *tick,
                    const int32_t *vox, float *t_arrival, void *stream);

/* The whole light path for one event after sim_quench_drift: yield,
 * photocurrent, scintillation, fluctuation and electronics, intermediates in
 * the workspace (sim_light_workspace_size); wave as above. */
int sim_light_workspace_size(const sim_config *cfg, const sim_light_config *lc, int64_t n_segments,
                             size_t *bytes);
int sim_light_event(const sim_config *cfg, const sim_light_config *lc, const sim_segments *seg,
                    const sim_drifted *dr, uint16_t *wave, void *ws, size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LARPIX_GB300_SIM_H */
