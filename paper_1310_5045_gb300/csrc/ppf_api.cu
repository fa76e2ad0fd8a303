// ppf_api.cu -- the C ABI of include/ppf.h: context life cycle, argument
// checks, the step / resample state machine and the host side of every call.
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "ppf_device.cuh"
#include "ppf_internal.h"

using namespace ppf;

namespace {

void set_err(ppf_ctx *c, const char *fmt, ...)
{
    if (!c)
        return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
}

// Host-side fault injection: PPF_FAULT=alloc makes ppf_create fail as if the
// device allocation failed, PPF_FAULT=launch makes ppf_step fail as if the
// launch failed, PPF_FAULT=timeout makes ppf_estimate report the timeout flag
// as if a bounded device wait had given up.  No GPU fault is ever produced.
bool fault(const char *what)
{
    const char *f = getenv("PPF_FAULT");
    return f && strcmp(f, what) == 0;
}

ppf_status cuda_fail(ppf_ctx *c, cudaError_t e, const char *where)
{
    set_err(c, "%s: %s", where, cudaGetErrorString(e));
    return PPF_ECUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess)                                \
            return cuda_fail(c, e_, #call);                   \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0)
        count = 1;
    return cudaMalloc((void **)p, sizeof(T) * count);
}

void free_all(ppf_ctx *c)
{
    void *ptrs[] = {c->tang[0], c->tang[1], c->gpart,
                    c->state[0], c->state[1], c->anc, c->anc_sys, c->lwp, c->goff, c->goff_new, c->ring, c->succ, c->Zp,
                    c->frame_buf[0], c->frame_buf[1], c->lmap, c->part, c->sum, c->est_dev, c->sc.Qt, c->sc.Ct, c->sc.Tt, c->sc.item_off, c->sc.extra, c->sc.Cbl,
                    c->sc.Tg, c->sc.tile_g, c->sc.ggrid, c->sc.split, c->sc.skey, c->sc.sval, c->sc.seg_tick, c->sc.seg_dst, c->sc.seg_len,
                    c->sc.seg_chunk, c->bin_key, c->bin_l, c->bin_tot, c->bin_item, c->bin_rec};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    if (c->sum_host)
        cudaFreeHost(c->sum_host);
    if (c->ev_scan)
        cudaEventDestroy(c->ev_scan);
    if (c->ev_sched)
        cudaEventDestroy(c->ev_sched);
    if (c->side_stream)
        cudaStreamDestroy(c->side_stream);
    if (c->prof_ev) {
        for (int i = 0; i < 4 * 2 * c->prof_cap; ++i)
            cudaEventDestroy(c->prof_ev[i]);
        free(c->prof_ev);
    }
}

// the largest and smallest group of a layout into the device summary (the
// systematic resample keeps the layout and leaves them as they are)
cudaError_t store_group_extents(ppf_ctx *c, const int64_t *off)
{
    int64_t mx = 0, mn = INT64_MAX;
    for (int32_t g = 0; g < c->G; ++g) {
        const int64_t sz = off[g + 1] - off[g];
        mx = sz > mx ? sz : mx;
        mn = sz < mn ? sz : mn;
    }
    const int64_t ext[2] = {mx, mn};
    static_assert(offsetof(DevSummary, min_group) == offsetof(DevSummary, max_group) + sizeof(int64_t),
                  "max_group and min_group are adjacent");
    cudaError_t e = cudaMemcpyAsync((char *)c->sum + offsetof(DevSummary, max_group), ext, sizeof(ext),
                                    cudaMemcpyHostToDevice, c->stream);
    return e == cudaSuccess ? cudaStreamSynchronize(c->stream) : e;
}

// the ARNA ring in group order (host copy, synchronous)
cudaError_t identity_ring(ppf_ctx *c)
{
    int32_t *h = (int32_t *)malloc(sizeof(int32_t) * (size_t)c->G);
    if (!h)
        return cudaErrorMemoryAllocation;
    for (int32_t g = 0; g < c->G; ++g)
        h[g] = g;
    cudaError_t e = cudaMemcpyAsync(c->ring, h, sizeof(int32_t) * (size_t)c->G, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    free(h);
    return e;
}

size_t dtype_size(int32_t dt)
{
    return dt == PPF_F32 ? 4 : 2;
}

}  // namespace

namespace ppf {
void prof_mark(ppf_ctx *c, int phase, int end)
{
    if (!c->prof_on)
        return;
    const int i = c->prof_n[phase];
    if (i >= c->prof_cap)
        return;
    cudaEventRecord(c->prof_ev[(phase * c->prof_cap + i) * 2 + end], c->stream);
    if (end)
        c->prof_n[phase] = i + 1;
}
}  // namespace ppf

extern "C" {

const char *ppf_status_string(ppf_status s)
{
    switch (s) {
    case PPF_OK: return "PPF_OK";
    case PPF_EINVAL: return "PPF_EINVAL: invalid argument";
    case PPF_ENOMEM: return "PPF_ENOMEM: out of memory";
    case PPF_ECUDA: return "PPF_ECUDA: CUDA runtime error";
    case PPF_ETIMEOUT: return "PPF_ETIMEOUT: device-side wait timed out";
    case PPF_EDEGENERATE: return "PPF_EDEGENERATE: all weights zero or NaN";
    case PPF_ESTATE: return "PPF_ESTATE: call out of order";
    }
    return "PPF_UNKNOWN";
}

const char *ppf_last_error(const ppf_ctx *ctx)
{
    return ctx ? ctx->err : "";
}

ppf_status ppf_create(const ppf_model *m, int64_t n, int32_t group_size, void *stream, ppf_ctx **out)
{
    if (!m || !out)
        return PPF_EINVAL;
    if (n < 1 || n > 2147483647LL || group_size < 1 || group_size > n)
        return PPF_EINVAL;
    if (m->width < 1 || m->height < 1 || m->patch_radius < 0 || m->patch_radius > MAX_RADIUS)
        return PPF_EINVAL;
    if (!(m->psf_sigma > 0.0f) || !(m->sigma_xi > 0.0f) || !(m->sigma_m >= 0.0f) || !(m->sigma_v >= 0.0f) ||
        !(m->sigma_I >= 0.0f) || !(m->v0_max >= 0.0f))
        return PPF_EINVAL;
    if (m->frame_dtype != PPF_F32 && m->frame_dtype != PPF_BF16 && m->frame_dtype != PPF_F16)
        return PPF_EINVAL;
    if (m->likelihood > 1)
        return PPF_EINVAL;
    if ((int64_t)(m->width + 4 * m->patch_radius) * (m->height + 4 * m->patch_radius) > (1LL << 31))
        return PPF_EINVAL;
    if (fault("alloc"))
        return PPF_ENOMEM;
    ppf_ctx *c = new (std::nothrow) ppf_ctx();
    if (!c)
        return PPF_ENOMEM;
    memset((void *)c, 0, sizeof(*c));
    c->m = *m;
    c->N = n;
    c->group_size = group_size;
    c->G = (int32_t)((n + group_size - 1) / group_size);
    c->T = (int32_t)((n + TILE - 1) / TILE);
    c->stream = (cudaStream_t)stream;
    c->pad = 2 * m->patch_radius;
    // row pitch (in pixel pairs): the padded width plus one zero column (the
    // frame is held as pairs (Z(col), Z(col + 1)), so that the patch sum reads
    // aligned pixel pairs), rounded up to even so that a row is a multiple of
    // 16 bytes (the tensor copies of the binned path need it)
    c->Wp = (m->width + 2 * c->pad + 2) & ~1;
    c->Hp = m->height + 2 * c->pad;
    c->frame_bytes = (size_t)m->width * m->height * dtype_size(m->frame_dtype);
    c->mode = MODE_CARRY;
    ppf_status st = PPF_OK;
    auto chk = [&](cudaError_t e, const char *w) {
        if (e != cudaSuccess && st == PPF_OK) {
            st = (e == cudaErrorMemoryAllocation) ? PPF_ENOMEM : PPF_ECUDA;
            set_err(c, "%s: %s", w, cudaGetErrorString(e));
        }
    };
    chk(cudaGetDevice(&c->device), "cudaGetDevice");
    if (st == PPF_OK)
        chk(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device), "attr");
    const int64_t N = n, G = c->G, T = c->T;
    if (st == PPF_OK) {
        chk(dalloc(&c->state[0], 6 * N), "state0");
        chk(dalloc(&c->state[1], 6 * N), "state1");
        chk(dalloc(&c->anc, N), "anc");
        chk(dalloc(&c->anc_sys, N), "anc_sys");
        chk(dalloc(&c->lwp, N), "lwp");
        chk(dalloc(&c->goff, G + 1), "goff");
        chk(dalloc(&c->goff_new, G + 1), "goff_new");
        chk(dalloc(&c->ring, G), "ring");
        chk(dalloc(&c->succ, G), "ring successors");
        chk(dalloc(&c->Zp, 2 * (size_t)c->Wp * c->Hp), "Zp");
        if (m->likelihood == 1)
            chk(dalloc(&c->lmap, (size_t)(m->width + 2 * m->patch_radius) * (m->height + 2 * m->patch_radius)),
                "cell map");
        chk(dalloc((char **)&c->frame_buf[0], c->frame_bytes), "frame_buf");
        chk(dalloc((char **)&c->frame_buf[1], c->frame_bytes), "frame_buf");
        c->n_part = c->num_sms > 0 ? ppf::step_grid(c) : 1;
        chk(dalloc(&c->part, c->n_part), "partials");
        chk(dalloc(&c->sum, 1), "summary");
        chk(dalloc(&c->est_dev, 1), "estimate staging");
        chk(dalloc(&c->sc.Qt, T), "Qt");
        chk(dalloc(&c->sc.Ct, T + 1), "Ct");
        chk(dalloc(&c->sc.Tt, T + 1), "Tt");
        chk(dalloc(&c->sc.item_off, T + 1), "item_off");
        chk(dalloc(&c->sc.extra, 2 * (N / ppf::ITEM_TICKETS + 1)), "further runs");
        chk(dalloc(&c->sc.Cbl, G + 1), "Cbl");
        chk(dalloc(&c->sc.Tg, G + 1), "Tg");
        chk(dalloc(&c->sc.tile_g, 2 * T), "tile groups");
        chk(dalloc(&c->sc.ggrid, G), "group draws");
        chk(dalloc(&c->sc.split, 4 * (T + G + 2 * (N / ppf::ITEM_TICKETS) + 2)), "split items");
        chk(dalloc(&c->sc.skey, 2 * G), "skey");
        chk(dalloc(&c->sc.sval, 5 * G), "sval");
        chk(dalloc(&c->sc.seg_tick, 2 * G + 1), "seg_tick");
        chk(dalloc(&c->sc.seg_dst, 2 * G + 1), "seg_dst");
        chk(dalloc(&c->sc.seg_len, 2 * G + 1), "seg_len");
        chk(dalloc(&c->sc.seg_chunk, 2 * G + 2), "seg_chunk");
        chk(cudaMallocHost((void **)&c->sum_host, sizeof(DevSummary)), "sum_host");
        {   // the side stream at the highest priority: its one-block schedule is
            // dispatched before the fill's blocks fill the SMs
            int lo = 0, hi = 0;
            chk(cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
            chk(cudaStreamCreateWithPriority(&c->side_stream, cudaStreamNonBlocking, hi), "side stream");
        }
        chk(cudaEventCreateWithFlags(&c->ev_scan, cudaEventDisableTiming), "event");
        chk(cudaEventCreateWithFlags(&c->ev_sched, cudaEventDisableTiming), "event");
    }
    if (st == PPF_OK) {
        chk(cudaMemsetAsync(c->sum, 0, sizeof(DevSummary), c->stream), "memset summary");
        // balanced group offsets
        int64_t *h = (int64_t *)malloc(sizeof(int64_t) * (G + 1));
        if (!h) {
            st = PPF_ENOMEM;
        } else {
            const int64_t base = N / G, extra = N % G;
            h[0] = 0;
            for (int64_t g = 0; g < G; ++g)
                h[g + 1] = h[g] + base + (g < extra ? 1 : 0);
            chk(cudaMemcpy(c->goff, h, sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice), "goff");
            if (st == PPF_OK)
                chk(store_group_extents(c, h), "group extents");
            free(h);
        }
    }
    if (st == PPF_OK)
        chk(identity_ring(c), "ring");
    if (st == PPF_OK)
        chk(ppf::resample_kernel_attributes(), "kernel attributes");
    c->bin_force = -1;
    if (st == PPF_OK)
        chk(ppf::bin_setup(c), "binned likelihood path");
    if (st == PPF_OK)
        chk(ppf::launch_init(c), "init_kernel");
    if (st == PPF_OK)
        chk(ppf::launch_identity(c, c->anc), "identity");
    if (st != PPF_OK) {
        if (getenv("PPF_VERBOSE"))
            fprintf(stderr, "ppf_create: %s\n", c->err);
        free_all(c);
        delete c;
        return st;
    }
    *out = c;
    return PPF_OK;
}

void ppf_destroy(ppf_ctx *c)
{
    if (!c)
        return;
    cudaStreamSynchronize(c->stream);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        for (int b = 0; b < 2; ++b) {
            cudaEventDestroy(c->fb_copied[b]);
            cudaEventDestroy(c->fb_free[b]);
        }
        cudaStreamDestroy(c->copy_stream);
    }
    free_all(c);
    delete c;
}

ppf_status ppf_step(ppf_ctx *c, const void *frame_dev, int32_t k)
{
    const ppf::NvtxRange nvtx_range("ppf_step");
    if (!c || !frame_dev || k < 1)
        return PPF_EINVAL;
    if (fault("launch")) {
        set_err(c, "injected launch failure");
        return PPF_ECUDA;
    }
    CK(ppf::launch_prepare_frame(c, frame_dev));
    CK(ppf::launch_step(c, k));
    c->n_steps += 1;
    c->cur ^= 1;
    c->mode = MODE_CARRY;
    c->stepped = true;
    c->weighted = true;
    c->last_frame = k;
    return PPF_OK;
}

// The frame is copied on a second stream into one of two device buffers, so
// the copy of frame k+1 overlaps the kernels of frame k: the step waits for
// its copy (event), and a buffer is refilled only after the step that read it.
ppf_status ppf_step_host(ppf_ctx *c, const void *frame_host, int32_t k)
{
    const ppf::NvtxRange nvtx_range("ppf_step_host");
    if (!c || !frame_host || k < 1)
        return PPF_EINVAL;
    if (!c->copy_stream) {
        CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            CK(cudaEventCreateWithFlags(&c->fb_copied[b], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&c->fb_free[b], cudaEventDisableTiming));
        }
    }
    const int b = c->fb_next;
    if (c->fb_used[b])
        CK(cudaStreamWaitEvent(c->copy_stream, c->fb_free[b], 0));
    CK(cudaMemcpyAsync(c->frame_buf[b], frame_host, c->frame_bytes, cudaMemcpyHostToDevice, c->copy_stream));
    CK(cudaEventRecord(c->fb_copied[b], c->copy_stream));
    CK(cudaStreamWaitEvent(c->stream, c->fb_copied[b], 0));
    c->h2d_bytes += (int64_t)c->frame_bytes;
    const ppf_status st = ppf_step(c, c->frame_buf[b], k);
    CK(cudaEventRecord(c->fb_free[b], c->stream));
    c->fb_used[b] = true;
    c->fb_next = b ^ 1;
    return st;
}

ppf_status ppf_resample(ppf_ctx *c, ppf_scheme scheme, float alpha)
{
    return ppf_resample_if(c, scheme, alpha, INFINITY);
}

ppf_status ppf_resample_if(ppf_ctx *c, ppf_scheme scheme, float alpha, double ess_threshold)
{
    const ppf::NvtxRange nvtx_range("ppf_resample");
    if (!c)
        return PPF_EINVAL;
    if (ess_threshold != ess_threshold)  // NaN
        return PPF_EINVAL;
    if (scheme < PPF_SYSTEMATIC || scheme > PPF_ARNA)
        return PPF_EINVAL;
    if ((scheme == PPF_RNA || scheme == PPF_ARNA) && !(alpha >= 0.0f && alpha <= 1.0f))
        return PPF_EINVAL;
    const bool sorted_groups = (scheme >= PPF_RPA_GS && scheme <= PPF_RPA_LGS) ||
                               (scheme >= PPF_RPA2_GS && scheme <= PPF_RPA2_LGS) || scheme == PPF_ARNA;
    if (sorted_groups && c->G > MAX_SCHED_GROUPS) {
        set_err(c, "RPA schedules and the ARNA ring support at most %d groups", MAX_SCHED_GROUPS);
        return PPF_EINVAL;
    }
    if (!c->weighted)
        return PPF_ESTATE;
    if (scheme == PPF_RNA || scheme == PPF_ARNA) {
        CK(scheme == PPF_RNA ? ppf::launch_resample_rna(c, alpha, ess_threshold)
                             : ppf::launch_resample_arna(c, alpha, ess_threshold));
        c->mode = MODE_EXPLICIT;
    } else {
        CK(ppf::launch_resample_global(c, (int)scheme, ess_threshold));
        if (scheme != PPF_SYSTEMATIC) {
            int64_t *t = c->goff;
            c->goff = c->goff_new;
            c->goff_new = t;
        }
        c->mode = MODE_UNIFORM;
    }
    c->weighted = false;
    c->n_resamples += 1;
    return PPF_OK;
}

ppf_status ppf_estimate(ppf_ctx *c, ppf_estimate_t *out)
{
    const ppf::NvtxRange nvtx_range("ppf_estimate");
    if (!c || !out)
        return PPF_EINVAL;
    if (!c->stepped)
        return PPF_ESTATE;
    CK(cudaMemcpyAsync(c->sum_host, c->sum, sizeof(DevSummary), cudaMemcpyDeviceToHost, c->stream));
    c->d2h_bytes += (int64_t)sizeof(DevSummary);
    CK(cudaStreamSynchronize(c->stream));
    const DevSummary &s = *c->sum_host;
    const int32_t flags = s.flags | (fault("timeout") ? FLAG_TIMEOUT : 0);
    for (int i = 0; i < 5; ++i)
        out->mean[i] = s.mean[i];
    out->log_evidence = s.log_evidence;
    out->ess = s.ess;
    out->max_log_weight = s.max_lw;
    out->frame = s.frame;
    out->status_flags = flags;
    out->links = s.links;
    out->moved = s.moved;
    out->max_group = s.max_group;
    out->min_group = s.min_group;
    if (flags) {
        if (s.flags) {
            const int32_t zero = 0;
            CK(cudaMemcpyAsync((char *)c->sum + offsetof(DevSummary, flags), &zero, sizeof(zero),
                               cudaMemcpyHostToDevice, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        if (flags & (FLAG_INTERNAL | FLAG_BAD_ANCESTOR)) {
            set_err(c, "device flags 0x%x: %s", flags,
                    (flags & FLAG_BAD_ANCESTOR)
                        ? "ancestor index out of range (treated as identity)"
                        : "internal consistency check failed (routing schedule, or an index check of the "
                          "debug build); the access was skipped");
            return PPF_EINVAL;
        }
        if (flags & FLAG_DEGENERATE)
            return PPF_EDEGENERATE;
        if (flags & FLAG_TIMEOUT)
            return PPF_ETIMEOUT;
    }
    return PPF_OK;  // FLAG_KEPT (N_eff test) and FLAG_RING (ARNA redraw) are information, not errors
}

ppf_status ppf_estimate_async(ppf_ctx *c, ppf_estimate_t *out)
{
    if (!c || !out)
        return PPF_EINVAL;
    if (!c->stepped)
        return PPF_ESTATE;
    CK(ppf::launch_format_estimate(c));
    CK(cudaMemcpyAsync(out, c->est_dev, sizeof(ppf_estimate_t), cudaMemcpyDeviceToHost, c->stream));
    c->d2h_bytes += (int64_t)sizeof(ppf_estimate_t);
    return PPF_OK;
}

ppf_status ppf_get_particles(ppf_ctx *c, float *state_dev, int32_t *anc_dev, float *lwp_dev)
{
    if (!c)
        return PPF_EINVAL;
    if (state_dev)
        CK(cudaMemcpyAsync(state_dev, c->state[c->cur], sizeof(float) * 6 * c->N, cudaMemcpyDeviceToDevice,
                           c->stream));
    if (anc_dev || lwp_dev)
        CK(ppf::launch_pending(c, anc_dev, lwp_dev));
    return PPF_OK;
}

ppf_status ppf_set_particles(ppf_ctx *c, const float *state_dev, const int32_t *anc_dev, const float *lwp_dev)
{
    if (!c || !state_dev)
        return PPF_EINVAL;
    CK(cudaMemcpyAsync(c->state[c->cur], state_dev, sizeof(float) * 6 * c->N, cudaMemcpyDeviceToDevice,
                       c->stream));
    if (anc_dev)
        CK(cudaMemcpyAsync(c->anc, anc_dev, sizeof(int32_t) * c->N, cudaMemcpyDeviceToDevice, c->stream));
    else
        CK(ppf::launch_identity(c, c->anc));
    if (lwp_dev) {
        CK(cudaMemcpyAsync(c->lwp, lwp_dev, sizeof(float) * c->N, cudaMemcpyDeviceToDevice, c->stream));
        c->mode = MODE_EXPLICIT;
    } else {
        c->mode = anc_dev ? MODE_UNIFORM : MODE_CARRY;
    }
    const int32_t zero = 0;
    CK(cudaMemcpyAsync((char *)c->sum + offsetof(DevSummary, degenerate), &zero, sizeof(zero),
                       cudaMemcpyHostToDevice, c->stream));
    // particles of unknown spread: the next step bins them (and measures)
    CK(ppf::bin_set_next(c, 1));
    c->weighted = false;
    return PPF_OK;
}

ppf_status ppf_set_likelihood_path(ppf_ctx *c, int32_t path)
{
    if (!c || path < PPF_PATH_AUTO || path > PPF_PATH_BINNED)
        return PPF_EINVAL;
    if (path == PPF_PATH_BINNED && !c->bin_key) {
        set_err(c, "the binned likelihood path is not available for this context (pcSIR, or a frame too large)");
        return PPF_EINVAL;
    }
    c->bin_force = path == PPF_PATH_AUTO ? -1 : (path == PPF_PATH_BINNED ? 1 : 0);
    return PPF_OK;
}

ppf_status ppf_get_likelihood_path(ppf_ctx *c, int32_t *last_step_binned)
{
    if (!c || !last_step_binned)
        return PPF_EINVAL;
    int32_t v = 0;
    CK(cudaMemcpyAsync(&v, (char *)c->sum + offsetof(DevSummary, bin_this), sizeof(v), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *last_step_binned = c->bin_key ? v : 0;
    return PPF_OK;
}

ppf_status ppf_get_groups(ppf_ctx *c, int32_t *n_groups, int64_t *offsets_host)
{
    if (!c)
        return PPF_EINVAL;
    if (n_groups)
        *n_groups = c->G;
    if (offsets_host) {
        CK(cudaMemcpyAsync(offsets_host, c->goff, sizeof(int64_t) * (c->G + 1), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return PPF_OK;
}

ppf_status ppf_set_groups(ppf_ctx *c, const int64_t *offsets_host)
{
    if (!c || !offsets_host)
        return PPF_EINVAL;
    if (offsets_host[0] != 0 || offsets_host[c->G] != c->N)
        return PPF_EINVAL;
    for (int32_t g = 0; g < c->G; ++g)
        if (offsets_host[g + 1] < offsets_host[g])
            return PPF_EINVAL;
    CK(cudaMemcpyAsync(c->goff, offsets_host, sizeof(int64_t) * (c->G + 1), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));  // offsets_host may be released on return
    CK(store_group_extents(c, offsets_host));
    CK(identity_ring(c));
    return PPF_OK;
}

ppf_status ppf_get_ring(ppf_ctx *c, int32_t *ring_host)
{
    if (!c || !ring_host)
        return PPF_EINVAL;
    CK(cudaMemcpyAsync(ring_host, c->ring, sizeof(int32_t) * (size_t)c->G, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PPF_OK;
}

ppf_status ppf_set_ring(ppf_ctx *c, const int32_t *ring_host)
{
    if (!c || !ring_host)
        return PPF_EINVAL;
    unsigned char *seen = (unsigned char *)calloc((size_t)c->G, 1);
    if (!seen)
        return PPF_ENOMEM;
    bool ok = true;
    for (int32_t p = 0; p < c->G && ok; ++p) {
        const int32_t g = ring_host[p];
        ok = g >= 0 && g < c->G && !seen[g];
        if (ok)
            seen[g] = 1;
    }
    free(seen);
    if (!ok)
        return PPF_EINVAL;
    CK(cudaMemcpyAsync(c->ring, ring_host, sizeof(int32_t) * (size_t)c->G, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PPF_OK;
}

ppf_status ppf_profile_enable(ppf_ctx *c, int enable, int32_t capacity)
{
    if (!c || (enable && capacity < 1))
        return PPF_EINVAL;
    if (!enable) {
        c->prof_on = false;
        return PPF_OK;
    }
    if (c->prof_ev && c->prof_cap < capacity) {
        CK(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < 4 * 2 * c->prof_cap; ++i)
            cudaEventDestroy(c->prof_ev[i]);
        free(c->prof_ev);
        c->prof_ev = nullptr;
    }
    if (!c->prof_ev) {
        c->prof_ev = (cudaEvent_t *)calloc((size_t)8 * capacity, sizeof(cudaEvent_t));
        if (!c->prof_ev)
            return PPF_ENOMEM;
        c->prof_cap = capacity;
        for (int i = 0; i < 8 * capacity; ++i)
            CK(cudaEventCreate(&c->prof_ev[i]));
    }
    CK(cudaStreamSynchronize(c->stream));
    for (int p = 0; p < 4; ++p)
        c->prof_n[p] = 0;
    c->launches = c->n_steps = c->n_resamples = c->h2d_bytes = c->d2h_bytes = 0;
    c->prof_on = true;
    return PPF_OK;
}

ppf_status ppf_profile_read(ppf_ctx *c, ppf_profile_t *out)
{
    if (!c || !out)
        return PPF_EINVAL;
    memset(out, 0, sizeof(*out));
    out->launches = c->launches;
    out->steps = c->n_steps;
    out->resamples = c->n_resamples;
    out->h2d_bytes = c->h2d_bytes;
    out->d2h_bytes = c->d2h_bytes;
    if (!c->prof_ev)
        return PPF_OK;
    CK(cudaStreamSynchronize(c->stream));
    double ms[4] = {0, 0, 0, 0};
    for (int p = 0; p < 4; ++p)
        for (int i = 0; i < c->prof_n[p]; ++i) {
            float t = 0.0f;
            CK(cudaEventElapsedTime(&t, c->prof_ev[(p * c->prof_cap + i) * 2], c->prof_ev[(p * c->prof_cap + i) * 2 + 1]));
            ms[p] += t;
        }
    out->prepare_ms = ms[PH_PREPARE];
    out->step_ms = ms[PH_STEP];
    out->finalize_ms = ms[PH_FINALIZE];
    out->resample_ms = ms[PH_RESAMPLE];
    out->timed_steps = c->prof_n[PH_STEP];
    return PPF_OK;
}

ppf_status ppf_loglik_grad(ppf_ctx *c, const void *frames_dev, int32_t K, const float *theta, double *loglik,
                           double *grad, int32_t *anc_dev, int32_t *anchors_dev)
{
    const ppf::NvtxRange nvtx_range("ppf_loglik_grad");
    if (c && c->m.likelihood != 0) {
        set_err(c, "ppf_loglik_grad needs the eq. 4 likelihood (model.likelihood = 0)");
        return PPF_EINVAL;
    }
    if (!c || !frames_dev || K < 1 || !loglik || !grad)
        return PPF_EINVAL;
    if (theta && !(theta[0] > 0.0f && theta[3] >= 0.0f))
        return PPF_EINVAL;
    const int64_t N = c->N;
    if (!c->tang[0]) {
        cudaError_t e1 = cudaMalloc((void **)&c->tang[0], sizeof(float) * 2 * N);
        cudaError_t e2 = cudaMalloc((void **)&c->tang[1], sizeof(float) * 2 * N);
        cudaError_t e3 = cudaMalloc((void **)&c->gpart, sizeof(GradPartial) * c->n_part);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            set_err(c, "gradient buffers: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3));
            return PPF_ENOMEM;
        }
    }
    const ppf_model saved = c->m;
    if (theta) {
        c->m.psf_sigma = theta[0];
        c->m.amplitude = theta[1];
        c->m.background = theta[2];
        c->m.sigma_m = theta[3];
    }
    ppf_status st = PPF_OK;
    auto run = [&]() -> ppf_status {
        CK(cudaMemsetAsync((char *)c->sum + offsetof(DevSummary, grad_L), 0, sizeof(double) * 5, c->stream));
        CK(cudaMemsetAsync((char *)c->sum + offsetof(DevSummary, degenerate), 0, sizeof(int32_t), c->stream));
        CK(cudaMemsetAsync((char *)c->sum + offsetof(DevSummary, flags), 0, sizeof(int32_t), c->stream));
        CK(ppf::launch_init(c));
        c->launches += 1;
        const char *fr = (const char *)frames_dev;
        for (int32_t k = 1; k <= K; ++k) {
            if (anc_dev) {
                if (k == 1)
                    CK(ppf::launch_identity(c, anc_dev));
                else
                    CK(cudaMemcpyAsync(anc_dev + (int64_t)(k - 1) * N, c->anc, sizeof(int32_t) * N,
                                       cudaMemcpyDeviceToDevice, c->stream));
            }
            CK(ppf::launch_prepare_frame(c, fr + (size_t)(k - 1) * c->frame_bytes));
            prof_mark(c, PH_STEP, 0);
            CK(ppf::launch_grad_step(c, k, k == 1, anchors_dev ? anchors_dev + (int64_t)(k - 1) * 2 * N : nullptr));
            prof_mark(c, PH_STEP, 1);
            c->cur ^= 1;
            c->tcur ^= 1;
            c->last_frame = k;
            c->n_steps += 1;
            if (k < K) {
                CK(ppf::launch_resample_global(c, PPF_SYSTEMATIC, INFINITY));
                c->n_resamples += 1;
            }
        }
        CK(cudaMemcpyAsync(c->sum_host, c->sum, sizeof(DevSummary), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return PPF_OK;
    };
    st = run();
    c->m = saved;
    c->mode = MODE_CARRY;
    c->stepped = true;
    c->weighted = true;
    if (st != PPF_OK)
        return st;
    *loglik = c->sum_host->grad_L;
    for (int q = 0; q < 4; ++q)
        grad[q] = c->sum_host->grad_g[q];
    return (c->sum_host->flags & FLAG_DEGENERATE) ? PPF_EDEGENERATE : PPF_OK;
}

}  // extern "C"
