// api.cu -- the C ABI of include/sim.h: host-side argument checks, workspace
// layout and the asynchronous enqueue of the path's kernels on the caller's
// stream.  Nothing here allocates device memory or synchronises the host.
#include <string.h>

#include "sim_internal.cuh"

using namespace larsim;

namespace {

thread_local int g_last_cuda = 0;

int cuda_fail(cudaError_t e)
{
    g_last_cuda = (int)e;
    return SIM_ERR_CUDA;
}

bool cfg_ok(const sim_config *c)
{
    if (!c) return false;
    if (c->n_mod_x < 1 || c->n_mod_y < 1 || (c->n_tpc != 1 && c->n_tpc != 2)) return false;
    if (c->tiles_x < 1 || c->tiles_y < 1 || c->px_per_tile < 1) return false;
    const int64_t npx = (int64_t)c->n_mod_x * c->n_mod_y * c->n_tpc * c->tiles_x * c->px_per_tile *
                        c->tiles_y * c->px_per_tile;
    if (npx >= ((int64_t)1 << 31)) return false;
    if (!(c->pitch_cm > 0.f) || !(c->drift_len_cm > 0.f) || !(c->vdrift_cm_us > 0.f)) return false;
    if (!(c->tick_us > 0.f) || c->n_ticks < 1 || !(c->sample_step_cm > 0.f)) return false;
    if (c->mc_per_sample < 1 || !(c->diff_clip_sigma >= 0.f) || !(c->lifetime_us > 0.f)) return false;
    if (c->recomb_model != 0 && c->recomb_model != 1) return false;
    if (c->adc_bits < 1 || c->adc_bits > 16 || c->hold_ticks < 0 || c->min_adc_interval_ticks < 0) return false;
    if (c->periodic_reset_ticks < 0 || c->precision < 0 || c->precision > 3) return false;
    if (c->fp64_charge != 0 && c->fp64_charge != 1) return false;
    if (c->per_point_drift != 0 && c->per_point_drift != 1) return false;
    if (c->nearest_lut != 0 && c->nearest_lut != 1) return false;
    if (c->tc_units_per_sm < 0 || c->tc_units_per_sm > 16) return false;
    if (c->tc_record_chunk != 0 && (c->tc_record_chunk < 4096 || c->tc_record_chunk > (1 << 20) ||
                                    (c->tc_record_chunk & (c->tc_record_chunk - 1)) != 0))
        return false;
    if (c->direct_ctas_per_sm < 0 || c->direct_ctas_per_sm > 4) return false;
    if (c->wait_spin_limit < 0 || c->wait_spin_limit > (1 << 30)) return false;
    return true;
}

bool events_ok(const sim_config *c, const sim_segments *s)
{
    if (!s || s->n_events < 0) return false;
    if (s->n_events > 0 && (!s->event_offsets || !s->event_ids)) return false;
    const int64_t slots = s->n_events > 0 ? s->n_events : 1;
    return detector_pixels(geo_of(*c)) * slots < ((int64_t)1 << 31);
}

bool seg_ok(const sim_segments *s)
{
    if (!s || s->n < 0 || s->n >= ((int64_t)1 << 31)) return false;
    if (s->n_events < 0 || (s->n_events > 0 && (!s->event_offsets || !s->event_ids))) return false;
    if (s->n == 0) return true;
    return s->x0 && s->y0 && s->z0 && s->t0 && s->x1 && s->y1 && s->z1 && s->t1 && s->dE;
}

bool resp_ok(const sim_response *r, bool need_table)
{
    if (!r || r->nb < 1 || r->nt < 1 || r->ld < r->nt || (r->ld % 4) != 0 || r->bins_per_pitch < 1) return false;
    if (!current_table_ok(r->nb, r->nt)) return false;
    if (need_table && (!r->lut || (reinterpret_cast<uintptr_t>(r->lut) & 15) != 0)) return false;
    return true;
}

bool drifted_ok(const sim_drifted *d)
{
    return d && d->Qa && d->t_drift && d->sigma_T && d->sigma_L && d->anode && d->n_samples && d->anchors &&
           (reinterpret_cast<uintptr_t>(d->anchors) & 15) == 0;
}

bool hits_ok(const sim_hits *h)
{
    return h && h->capacity >= 0 && (h->capacity == 0 || (h->pixel && h->t_cross && h->t_adc && h->adc && h->q));
}

// Scratch and launch of the induced-current form selected by cfg.precision.
size_t current_scratch(const sim_config &c, int64_t pixels)
{
    if (c.precision == 3) return current_direct_scratch_bytes(pixels);
    return c.precision == 0 ? current_scratch_bytes(pixels)
                            : current_tc_scratch_bytes(pixels, c.n_ticks, c.tc_units_per_sm, c.tc_record_chunk);
}

cudaError_t launch_current(const sim_config &c, const sim_segments &s, const sim_drifted &d, const sim_response &r,
                           const int32_t *active, const int32_t *off, const int32_t *ids, const int64_t *counts,
                           int64_t pix_cap, float *current, void *scratch, cudaStream_t st,
                           int64_t pix_begin = 0, int64_t pix_end = INT64_MAX)
{
    if (c.precision == 0)
        return launch_induced_current(c, s, d, r, active, off, ids, counts, pix_cap, pix_begin, pix_end, current,
                                      scratch, st);
    if (c.precision == 3)
        return launch_induced_current_direct(c, s, d, r, active, off, ids, counts, pix_cap, pix_begin, pix_end,
                                             current, scratch, st);
    return launch_induced_current_tc(c, s, d, r, active, off, ids, counts, pix_cap, pix_begin, pix_end, current,
                                     scratch, st);
}

// Layout of sim_event's workspace.
struct Layout {
    size_t counts, scratch, Qa, td, sT, sL, anode, ns, anch;
    size_t seg_off, seg_ids, active, pix_off, pix_ids, current, total;
};

Layout layout(const sim_config &c, int64_t slots, int64_t n, int64_t pairs, int64_t pixels)
{
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    L.counts = take(256);
    size_t sc = map_scratch_bytes(c, n, slots);
    const size_t es = elec_scratch_bytes(c, pixels), cs = pixels > 0 ? current_scratch(c, pixels) : 0;
    if (es > sc) sc = es;
    if (cs > sc) sc = cs;
    L.scratch = take(sc);
    L.Qa = take(4 * (size_t)n);
    L.td = take(4 * (size_t)n);
    L.sT = take(4 * (size_t)n);
    L.sL = take(4 * (size_t)n);
    L.anode = take(4 * (size_t)n);
    L.ns = take(4 * (size_t)n);
    L.anch = take(SIM_ANCHOR_BYTES * (size_t)n);
    L.seg_off = take(4 * (size_t)(n + 1));
    L.seg_ids = take(4 * (size_t)pairs);
    L.active = take(4 * (size_t)pixels);
    L.pix_off = take(4 * (size_t)(pixels + 1));
    L.pix_ids = take(4 * (size_t)pairs);
    L.current = take(4 * (size_t)pixels * (size_t)c.n_ticks);
    L.total = o;
    return L;
}

void fill_view(const Layout &L, char *w, sim_event_view *v)
{
    v->dr.Qa = reinterpret_cast<float *>(w + L.Qa);
    v->dr.t_drift = reinterpret_cast<float *>(w + L.td);
    v->dr.sigma_T = reinterpret_cast<float *>(w + L.sT);
    v->dr.sigma_L = reinterpret_cast<float *>(w + L.sL);
    v->dr.anode = reinterpret_cast<int32_t *>(w + L.anode);
    v->dr.n_samples = reinterpret_cast<int32_t *>(w + L.ns);
    v->dr.anchors = w + L.anch;
    v->seg_pix_off = reinterpret_cast<int32_t *>(w + L.seg_off);
    v->seg_pix_ids = reinterpret_cast<int32_t *>(w + L.seg_ids);
    v->active_pixels = reinterpret_cast<int32_t *>(w + L.active);
    v->pix_seg_off = reinterpret_cast<int32_t *>(w + L.pix_off);
    v->pix_seg_ids = reinterpret_cast<int32_t *>(w + L.pix_ids);
    v->current = reinterpret_cast<float *>(w + L.current);
    v->counts = reinterpret_cast<int64_t *>(w + L.counts);
}

}  // namespace

namespace larsim {
// argument checks and error recording shared with pixel_map_static.cu
bool abi_config_ok(const sim_config *c) { return cfg_ok(c); }
bool abi_segments_ok(const sim_segments *s) { return seg_ok(s); }
bool abi_events_ok(const sim_config *c, const sim_segments *s) { return events_ok(c, s); }
bool abi_drifted_ok(const sim_drifted *d) { return drifted_ok(d); }
bool abi_response_ok(const sim_response *r, bool need_table) { return resp_ok(r, need_table); }
int abi_cuda_fail(cudaError_t e) { return cuda_fail(e); }
}  // namespace larsim

extern "C" {

const char *sim_strerror(int code)
{
    switch (code) {
    case SIM_OK: return "ok";
    case SIM_ERR_INVALID_ARG: return "invalid argument";
    case SIM_ERR_CAPACITY: return "capacity or workspace too small";
    case SIM_ERR_CUDA: return "CUDA error (see sim_last_cuda_error)";
    case SIM_ERR_TIMEOUT: return "device-side wait timed out";
    default: return "unknown error";
    }
}

int sim_last_cuda_error(void) { return g_last_cuda; }

void sim_abi_sizes(int64_t sizes[5])
{
    sizes[0] = sizeof(sim_config);
    sizes[1] = sizeof(sim_segments);
    sizes[2] = sizeof(sim_response);
    sizes[3] = sizeof(sim_drifted);
    sizes[4] = sizeof(sim_hits);
}

int sim_workspace_size(const sim_config *cfg, int64_t max_events, int64_t max_segments, int64_t max_pairs,
                       int64_t max_pixels, size_t *bytes)
{
    if (!cfg_ok(cfg) || !bytes || max_events < 0 || max_segments < 0 || max_pairs < 0 || max_pixels < 0)
        return SIM_ERR_INVALID_ARG;
    const int64_t slots = max_events > 0 ? max_events : 1;
    if (detector_pixels(geo_of(*cfg)) * slots >= ((int64_t)1 << 31)) return SIM_ERR_INVALID_ARG;
    *bytes = layout(*cfg, slots, max_segments, max_pairs, max_pixels).total;
    return SIM_OK;
}

const int64_t *sim_workspace_counts(const void *ws) { return reinterpret_cast<const int64_t *>(ws); }

int sim_quench_drift(const sim_config *cfg, const sim_segments *seg, const sim_drifted *out, void *stream)
{
    if (!cfg_ok(cfg) || !seg_ok(seg) || (seg->n > 0 && !drifted_ok(out))) return SIM_ERR_INVALID_ARG;
    const cudaError_t e = launch_quench_drift(*cfg, *seg, *out, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_pixel_map(const sim_config *cfg, const sim_segments *seg, const sim_drifted *dr,
                  const sim_response *resp, int32_t *seg_pix_off, int32_t *seg_pix_ids, int64_t pair_cap,
                  int32_t *active_pixels, int32_t *pix_seg_off, int32_t *pix_seg_ids, int64_t pix_cap,
                  void *ws, size_t ws_bytes, void *stream)
{
    if (!cfg_ok(cfg) || !seg_ok(seg) || !events_ok(cfg, seg) || !resp_ok(resp, false) || pair_cap < 0 ||
        pix_cap < 0 || !ws)
        return SIM_ERR_INVALID_ARG;
    if (seg->n > 0 && (!drifted_ok(dr) || !seg_pix_off)) return SIM_ERR_INVALID_ARG;
    if (!seg_pix_off || (pair_cap > 0 && (!seg_pix_ids || !pix_seg_ids)) ||
        (pix_cap > 0 && (!active_pixels || !pix_seg_off)) || (pix_cap == 0 && !pix_seg_off))
        return SIM_ERR_INVALID_ARG;
    if (ws_bytes < 256 + map_scratch_bytes(*cfg, seg->n, n_slots(events_of(*seg)))) return SIM_ERR_CAPACITY;
    char *w = reinterpret_cast<char *>(ws);
    const sim_drifted d0 = dr ? *dr : sim_drifted{};
    const cudaError_t e = launch_pixel_map(*cfg, *seg, d0, resp->nb, resp->bins_per_pitch, seg_pix_off,
                                           seg_pix_ids, pair_cap, active_pixels, pix_seg_off, pix_seg_ids,
                                           pix_cap, reinterpret_cast<int64_t *>(w), w + 256,
                                           (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_induced_current_range(const sim_config *cfg, const sim_segments *seg, const sim_drifted *dr,
                              const sim_response *resp, const int32_t *active_pixels, const int32_t *pix_seg_off,
                              const int32_t *pix_seg_ids, const int64_t *counts, int64_t pix_begin,
                              int64_t pix_end, int64_t pix_cap, float *current, void *ws, size_t ws_bytes,
                              void *stream)
{
    if (!cfg_ok(cfg) || !seg_ok(seg) || !events_ok(cfg, seg) || !resp_ok(resp, true) || !counts || pix_cap < 0 ||
        !ws || pix_begin < 0 || pix_end < pix_begin)
        return SIM_ERR_INVALID_ARG;
    if (pix_cap > 0 && (!active_pixels || !pix_seg_off || !pix_seg_ids || !current)) return SIM_ERR_INVALID_ARG;
    if (pix_cap > 0 && seg->n > 0 && !drifted_ok(dr)) return SIM_ERR_INVALID_ARG;
    if (pix_cap == 0 || pix_begin >= pix_cap || pix_end == pix_begin) return SIM_OK;
    if (ws_bytes < 256 + current_scratch(*cfg, pix_cap)) return SIM_ERR_CAPACITY;
    const sim_drifted d0 = dr ? *dr : sim_drifted{};
    const cudaError_t e = launch_current(*cfg, *seg, d0, *resp, active_pixels, pix_seg_off, pix_seg_ids, counts,
                                         pix_cap, current, reinterpret_cast<char *>(ws) + 256, (cudaStream_t)stream,
                                         pix_begin, pix_end);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_induced_current(const sim_config *cfg, const sim_segments *seg, const sim_drifted *dr,
                        const sim_response *resp, const int32_t *active_pixels, const int32_t *pix_seg_off,
                        const int32_t *pix_seg_ids, const int64_t *counts, int64_t pix_cap, float *current,
                        void *ws, size_t ws_bytes, void *stream)
{
    return sim_induced_current_range(cfg, seg, dr, resp, active_pixels, pix_seg_off, pix_seg_ids, counts, 0,
                                     INT64_MAX, pix_cap, current, ws, ws_bytes, stream);
}

int sim_electronics(const sim_config *cfg, const sim_segments *events, const int32_t *active_pixels,
                    const float *current, int64_t *counts, int64_t pix_cap, const sim_hits *out, void *ws,
                    size_t ws_bytes, void *stream)
{
    if (!cfg_ok(cfg) || !events_ok(cfg, events) || !counts || pix_cap < 0 || !hits_ok(out) || !ws)
        return SIM_ERR_INVALID_ARG;
    if (pix_cap > 0 && (!active_pixels || !current)) return SIM_ERR_INVALID_ARG;
    if (ws_bytes < 256 + elec_scratch_bytes(*cfg, pix_cap)) return SIM_ERR_CAPACITY;
    const cudaError_t e = launch_electronics(*cfg, events_of(*events), active_pixels, current, counts, pix_cap, *out,
                                             reinterpret_cast<char *>(ws) + 256, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_event_view_of(const sim_config *cfg, int64_t max_events, int64_t n_segments, int64_t max_pairs,
                      int64_t max_pixels, void *ws, size_t ws_bytes, sim_event_view *view)
{
    if (!cfg_ok(cfg) || max_events < 0 || n_segments < 0 || max_pairs < 0 || max_pixels < 0 || !ws || !view)
        return SIM_ERR_INVALID_ARG;
    const Layout L = layout(*cfg, max_events > 0 ? max_events : 1, n_segments, max_pairs, max_pixels);
    if (ws_bytes < L.total) return SIM_ERR_CAPACITY;
    fill_view(L, reinterpret_cast<char *>(ws), view);
    return SIM_OK;
}

int sim_event(const sim_config *cfg, const sim_segments *seg, const sim_response *resp, int64_t max_pairs,
              int64_t max_pixels, const sim_hits *out, void *ws, size_t ws_bytes, void *stream)
{
    if (!cfg_ok(cfg) || !seg_ok(seg) || !events_ok(cfg, seg) || !resp_ok(resp, true) || max_pairs < 0 ||
        max_pixels < 0 || !hits_ok(out) || !ws)
        return SIM_ERR_INVALID_ARG;
    const Layout L = layout(*cfg, n_slots(events_of(*seg)), seg->n, max_pairs, max_pixels);
    if (ws_bytes < L.total) return SIM_ERR_CAPACITY;
    char *w = reinterpret_cast<char *>(ws);
    sim_event_view v;
    fill_view(L, w, &v);
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_quench_drift(*cfg, *seg, v.dr, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_pixel_map(*cfg, *seg, v.dr, resp->nb, resp->bins_per_pitch, v.seg_pix_off, v.seg_pix_ids,
                         max_pairs, v.active_pixels, v.pix_seg_off, v.pix_seg_ids, max_pixels, v.counts,
                         w + L.scratch, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_current(*cfg, *seg, v.dr, *resp, v.active_pixels, v.pix_seg_off, v.pix_seg_ids, v.counts, max_pixels,
                       v.current, w + L.scratch, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_electronics(*cfg, events_of(*seg), v.active_pixels, v.current, v.counts, max_pixels, *out,
                           w + L.scratch, st);
    if (e != cudaSuccess) return cuda_fail(e);
    return SIM_OK;
}

int sim_response_cumulative(const sim_response *resp, float *cum, void *stream)
{
    if (!resp_ok(resp, true) || !cum || (reinterpret_cast<uintptr_t>(cum) & 15) != 0) return SIM_ERR_INVALID_ARG;
    const cudaError_t e = launch_response_cumulative(*resp, cum, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_hit_truth_workspace_size(int64_t max_hits, int64_t max_cells, size_t *bytes)
{
    if (max_hits < 0 || max_hits >= ((int64_t)1 << 31) || max_cells < 0 || max_cells >= ((int64_t)1 << 31) || !bytes)
        return SIM_ERR_INVALID_ARG;
    *bytes = hit_truth_workspace_bytes(max_hits, max_cells);
    return SIM_OK;
}

int sim_hit_truth(const sim_config *cfg, const sim_segments *seg, const sim_drifted *dr, const sim_response *resp,
                  const float *cum, const int32_t *active_pixels, const int32_t *pix_seg_off,
                  const int32_t *pix_seg_ids, const int64_t *counts, int64_t pix_cap, const sim_hits *hits,
                  const sim_truth *out, int64_t max_cells, void *ws, size_t ws_bytes, void *stream)
{
    if (!cfg_ok(cfg) || !seg_ok(seg) || !events_ok(cfg, seg) || !resp_ok(resp, false) || !cum || !counts ||
        pix_cap < 0 || !hits_ok(hits) || !hits->n_out || !out || !ws || max_cells < 0 ||
        max_cells >= ((int64_t)1 << 31) || (reinterpret_cast<uintptr_t>(cum) & 15) != 0)
        return SIM_ERR_INVALID_ARG;
    if (out->k < 1 || out->k > SIM_TRUTH_MAX_K || out->capacity < 0 || out->capacity >= ((int64_t)1 << 31))
        return SIM_ERR_INVALID_ARG;
    if (out->capacity > 0 && (!out->segment || !out->q || !out->q_signal)) return SIM_ERR_INVALID_ARG;
    if (pix_cap > 0 && (!active_pixels || !pix_seg_off || !pix_seg_ids)) return SIM_ERR_INVALID_ARG;
    if (seg->n > 0 && !drifted_ok(dr)) return SIM_ERR_INVALID_ARG;
    const int64_t hcap = hits->capacity < out->capacity ? hits->capacity : out->capacity;
    if (ws_bytes < hit_truth_workspace_bytes(hcap, max_cells)) return SIM_ERR_CAPACITY;
    const sim_drifted d0 = dr ? *dr : sim_drifted{};
    const cudaError_t e = launch_hit_truth(*cfg, *seg, d0, *resp, cum, active_pixels, pix_seg_off, pix_seg_ids,
                                           counts, pix_cap, *hits, *out, max_cells, ws, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_hit_points(const sim_config *cfg, const sim_hits *hits, const float *t_event, float *x, float *y, float *z,
                   void *stream)
{
    if (!cfg_ok(cfg) || !hits_ok(hits) || !hits->n_out) return SIM_ERR_INVALID_ARG;
    if (hits->capacity > 0 && (!x || !y || !z)) return SIM_ERR_INVALID_ARG;
    const cudaError_t e = launch_hit_points(*cfg, *hits, t_event, x, y, z, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_track_dqdx(const float *x, const float *y, const float *z, const float *q, const int64_t *n_points,
                   int64_t capacity, const double *origin, const double *direction, double piece_cm,
                   int32_t n_pieces, double r_max_cm, double *dq, int32_t *count, void *stream)
{
    if (!n_points || capacity < 0 || !origin || !direction || !(piece_cm > 0.0) || n_pieces < 1 ||
        !(r_max_cm >= 0.0) || !dq || !count)
        return SIM_ERR_INVALID_ARG;
    if (capacity > 0 && (!x || !y || !z || !q)) return SIM_ERR_INVALID_ARG;
    const cudaError_t e = launch_track_dqdx(x, y, z, q, n_points, capacity, origin, direction, piece_cm, n_pieces,
                                            r_max_cm, dq, count, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

static bool light_ok(const sim_config *c, const sim_light_config *lc)
{
    if (!cfg_ok(c) || !lc) return false;
    if (!lc->vis || !lc->tdist || !lc->eff || !lc->gain || !lc->resp || !lc->noise_amp) return false;
    if (lc->nvx < 1 || lc->nvy < 1 || lc->nvz < 1 || lc->n_det < 1 || lc->n_det > 32 || lc->nt < 1 || lc->nt > 256)
        return false;
    if (lc->n_resp < 1 || lc->n_resp > 2048 || lc->adc_bits < 1 || lc->adc_bits > 16) return false;
    if (lc->noise_block < 64 || lc->noise_block > 4096 || (lc->noise_block & (lc->noise_block - 1)) != 0) return false;
    if (!(lc->vox_cm > 0.f) || !(lc->w_ph_MeV > 0.f) || !(lc->tick_us > 0.f) || lc->n_ticks < 1) return false;
    if (!(lc->tau_fast_us > 0.f) || !(lc->tau_slow_us > 0.f) || !(lc->trunc_taus >= 0.f) || !(lc->sample_us > 0.f))
        return false;
    if (!(lc->fast_frac >= 0.f && lc->fast_frac <= 1.f)) return false;
    return (int64_t)light_n_det_total(*c, *lc) * lc->n_ticks < ((int64_t)1 << 40);
}

int sim_light_n_samples(const sim_light_config *lc, int64_t *n_samples)
{
    if (!lc || !n_samples || !(lc->sample_us > 0.f) || !(lc->tick_us > 0.f) || lc->n_ticks < 1)
        return SIM_ERR_INVALID_ARG;
    *n_samples = light_n_samples(*lc, nullptr);
    return SIM_OK;
}

int sim_light_yield(const sim_config *cfg, const sim_light_config *lc, const sim_segments *seg, const sim_drifted *dr,
                    float *npe, int32_t *tick, int32_t *vox, void *stream)
{
    if (!light_ok(cfg, lc) || !seg_ok(seg) || seg->n_events != 0) return SIM_ERR_INVALID_ARG;
    if (seg->n > 0 && (!drifted_ok(dr) || !npe || !tick || !vox)) return SIM_ERR_INVALID_ARG;
    const sim_drifted d0 = dr ? *dr : sim_drifted{};
    const cudaError_t e = launch_light_yield(*cfg, *lc, *seg, d0, npe, tick, vox, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_light_photocurrent(const sim_config *cfg, const sim_light_config *lc, const sim_segments *seg,
                           const sim_drifted *dr, const float *npe, const int32_t *tick, const int32_t *vox,
                           int64_t *pe_fix, void *stream)
{
    if (!light_ok(cfg, lc) || !seg_ok(seg) || seg->n_events != 0 || !pe_fix) return SIM_ERR_INVALID_ARG;
    if (seg->n > 0 && (!drifted_ok(dr) || !npe || !tick || !vox)) return SIM_ERR_INVALID_ARG;
    const sim_drifted d0 = dr ? *dr : sim_drifted{};
    const cudaError_t e = launch_light_photocurrent(*cfg, *lc, *seg, d0, npe, tick, vox, pe_fix, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_light_scintillation(const sim_config *cfg, const sim_light_config *lc, const int64_t *pe_fix, float *scint,
                            void *stream)
{
    if (!light_ok(cfg, lc) || !pe_fix || !scint) return SIM_ERR_INVALID_ARG;
    const cudaError_t e = launch_light_scint(*cfg, *lc, pe_fix, scint, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_light_fluctuate(const sim_config *cfg, const sim_light_config *lc, uint64_t event_id, const float *scint,
                        float *pe_obs, void *stream)
{
    if (!light_ok(cfg, lc) || !scint || !pe_obs) return SIM_ERR_INVALID_ARG;
    const cudaError_t e = launch_light_fluct(*cfg, *lc, event_id, scint, pe_obs, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_light_electronics(const sim_config *cfg, const sim_light_config *lc, uint64_t event_id, const float *pe_obs,
                          float *v, uint16_t *wave, void *stream)
{
    if (!light_ok(cfg, lc) || !pe_obs || !v || !wave) return SIM_ERR_INVALID_ARG;
    const cudaError_t e = launch_light_electronics(*cfg, *lc, event_id, pe_obs, v, wave, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

int sim_light_truth(const sim_config *cfg, const sim_light_config *lc, int64_t n_segments, const int32_t *tick,
                    const int32_t *vox, float *t_arrival, void *stream)
{
    if (!light_ok(cfg, lc) || n_segments < 0) return SIM_ERR_INVALID_ARG;
    if (n_segments > 0 && (!tick || !vox || !t_arrival)) return SIM_ERR_INVALID_ARG;
    const cudaError_t e = launch_light_truth(*lc, n_segments, tick, vox, t_arrival, (cudaStream_t)stream);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

namespace {
struct LightLayout {
    size_t npe, tick, vox, pe, scint, obs, v, total;
};
LightLayout light_layout(const sim_config &c, const sim_light_config &lc, int64_t n)
{
    LightLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    const size_t rows = (size_t)light_n_det_total(c, lc) * (size_t)lc.n_ticks;
    L.npe = take(4 * (size_t)n * lc.n_det);
    L.tick = take(4 * (size_t)n);
    L.vox = take(4 * (size_t)n);
    L.pe = take(8 * rows);
    L.scint = take(4 * rows);
    L.obs = take(4 * rows);
    L.v = take(4 * rows);
    L.total = o;
    return L;
}
}  // namespace

int sim_light_workspace_size(const sim_config *cfg, const sim_light_config *lc, int64_t n_segments, size_t *bytes)
{
    if (!light_ok(cfg, lc) || n_segments < 0 || !bytes) return SIM_ERR_INVALID_ARG;
    *bytes = light_layout(*cfg, *lc, n_segments).total;
    return SIM_OK;
}

int sim_light_event(const sim_config *cfg, const sim_light_config *lc, const sim_segments *seg, const sim_drifted *dr,
                    uint16_t *wave, void *ws, size_t ws_bytes, void *stream)
{
    if (!light_ok(cfg, lc) || !seg_ok(seg) || seg->n_events != 0 || !wave || !ws) return SIM_ERR_INVALID_ARG;
    if (seg->n > 0 && !drifted_ok(dr)) return SIM_ERR_INVALID_ARG;
    const LightLayout L = light_layout(*cfg, *lc, seg->n);
    if (ws_bytes < L.total) return SIM_ERR_CAPACITY;
    char *w = reinterpret_cast<char *>(ws);
    const cudaStream_t st = (cudaStream_t)stream;
    const sim_drifted d0 = dr ? *dr : sim_drifted{};
    float *npe = reinterpret_cast<float *>(w + L.npe);
    int32_t *tick = reinterpret_cast<int32_t *>(w + L.tick), *vox = reinterpret_cast<int32_t *>(w + L.vox);
    int64_t *pe = reinterpret_cast<int64_t *>(w + L.pe);
    float *scint = reinterpret_cast<float *>(w + L.scint), *obs = reinterpret_cast<float *>(w + L.obs);
    float *v = reinterpret_cast<float *>(w + L.v);
    cudaError_t e = launch_light_yield(*cfg, *lc, *seg, d0, npe, tick, vox, st);
    if (e == cudaSuccess) e = launch_light_photocurrent(*cfg, *lc, *seg, d0, npe, tick, vox, pe, st);
    if (e == cudaSuccess) e = launch_light_scint(*cfg, *lc, pe, scint, st);
    if (e == cudaSuccess) e = launch_light_fluct(*cfg, *lc, seg->event_id, scint, obs, st);
    if (e == cudaSuccess) e = launch_light_electronics(*cfg, *lc, seg->event_id, obs, v, wave, st);
    return e == cudaSuccess ? SIM_OK : cuda_fail(e);
}

}  // extern "C"
