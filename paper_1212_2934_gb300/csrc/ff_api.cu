// Host runtime and C interface of libff (declared in include/ff.h).
//
// A context owns its device memory and one stream.  The state lives on the
// GPU in two record buffers (positions, velocities, moments, angular
// velocities, particle ids) that alternate: the key sort gathers the state
// into Morton order in the other buffer, and the integrator writes the next
// state into the other buffer again.  Outputs go back to the caller's order
// through the particle ids.  Nothing crosses to the host inside a step.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

#include <algorithm>
#include <vector>
#include "ff.h"
#include "ffk.cuh"

namespace {

constexpr int64_t kMaxN = int64_t(1) << 27;

struct Buffers {
    void* pos = nullptr;
    void* vel = nullptr;
    void* u = nullptr;
    void* om = nullptr;
    uint32_t* id = nullptr;
};

}  // namespace

struct ff_ctx {
    ff_params p;
    int64_t n = 0;
    bool fp64 = false;
    bool mixed = false;  // single-precision tree with FP64 cell sums
    size_t rec = 16;  // bytes per record
    size_t cell_bytes = 32;  // bytes per Cell record
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t step = 0;
    bool have_particles = false;
    bool poisoned = false;
    char err[512] = {0};

    Buffers st[2];
    int cur = 0;
    uint64_t* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    uint32_t* radix_tmp = nullptr;
    uint32_t* cnt = nullptr;
    uint32_t* off = nullptr;
    uint32_t* scan_tmp = nullptr;
    ffk::BBox* bbox = nullptr;

    void* cell = nullptr;  // Cell<R> records: topology + centre
    void* mom = nullptr;
    void* lo = nullptr;
    void* sum = nullptr;
    ffk::dvec4* sum_hi = nullptr;  // FP64 cell sums (mixed precision only)
    void* q1 = nullptr;          // dipole-position terms per cell (quadrupole option only)
    void* q2 = nullptr;
    ffk::dvec4* mom_hi = nullptr;
    int* parent = nullptr;
    int* arrive = nullptr;
    int64_t cap = 0;

    void* h = nullptr;
    void* f = nullptr;
    void* esr = nullptr;
    int4* counts = nullptr;
    int* work = nullptr;         // traversal task counters
    double* partials = nullptr;
    double* obs = nullptr;       // observables of the last ff_energy
    double* obs_step = nullptr;  // observables of the state at the start of the last step
    unsigned long long* dstep = nullptr;  // device copy of the step counter (noise counter)
    // one captured step per starting state buffer (CUDA graphs)
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int gend[2] = {0, 0};           // state buffer after the captured step
    int64_t glaunch[2] = {0, 0};    // kernels in the captured step
    int* dflags = nullptr;
    int* hflags = nullptr;       // pinned mirror
    double* hobs = nullptr;      // pinned mirror of 10 doubles
    void* staging = nullptr;     // 4 x 3n doubles
    // energy gradient (allocated on first use; entry buffers grow as needed)
    uint32_t* e_cnt = nullptr;   // entries per particle (n)
    uint32_t* e_base = nullptr;  // their exclusive scan (n + 1)
    unsigned long long* e_total = nullptr;
    void* g_pos = nullptr;       // gradients in sorted order (records)
    void* g_u = nullptr;
    uint32_t* rs_key = nullptr;  // record space in each task's slots: source (e_cap)
    uint32_t* rs_mask = nullptr; //   lane mask; both also the record sort's second buffers
    uint32_t* e_tmp = nullptr;
    int64_t e_cap = 0;           // entries rs_key, rs_mask hold
    uint32_t* s_beg = nullptr;   // per source: entry range
    uint32_t* s_end = nullptr;
    double* s_G = nullptr;       // per source: 3 + 3 sums
    double* s_Q = nullptr;
    uint32_t* s_items = nullptr; // per source: work items of its entry list
    uint32_t* s_item_off = nullptr;
    uint32_t* s_scan = nullptr;
    int64_t s_cap = 0;           // sources the buffers hold
    double* i_part = nullptr;    // per work item: six partial sums; then each item's source
    int64_t i_cap = 0;
    // every particle's sources, written by the counting walk (chunks of kPoolChunk)
    uint32_t* p_keys = nullptr;
    uint32_t* p_link = nullptr;
    unsigned* p_next = nullptr;
    int64_t p_cap = 0;           // chunks
    uint32_t* s_src = nullptr;   // the source at each place of the depth-first order (s_cap)
    // records (one per task and source some particle of the task has)
    uint32_t* t_cnt = nullptr;   // per task: its records (ntask)
    uint32_t* t_off = nullptr;   // their exclusive scan (ntask + 1)
    uint32_t* s_rbeg = nullptr;  // per source: its first sorted record (s_cap)
    uint32_t* r_key = nullptr;   // packed in task order: the source
    uint32_t* r_idx = nullptr;   //   the packed index (sort value)
    uint2* r_rec = nullptr;      //   (task, lane mask)
    uint2* r_srec = nullptr;     // sorted by source
    uint32_t* r_E = nullptr;     //   entries before each sorted record (+1)
    unsigned long long* r_scan = nullptr;  // the one-pass scan's status words
    int64_t r_cap = 0;
    bool tree_valid = false;     // a Barnes-Hut tree of some state exists
    bool counts_valid = false;

    // batched ensembles (ff_set_systems); nsys = 0: one system with the context's field and box
    int nsys = 0;
    uint32_t* sys_of_pos = nullptr;  // device: system of each position
    int* sys_start = nullptr;        // device: nsys + 1 offsets
    void* sys_h = nullptr;           // device: vec4<R>[nsys] applied field
    void* sys_lo = nullptr;          // device: vec4<R>[nsys] lower wall planes
    void* sys_hi = nullptr;          // device: vec4<R>[nsys] upper wall planes
    double* sys_acc = nullptr;       // device: nsys x 4 sums of u and h_dip_z
    int64_t sys_steps = 0;           // steps accumulated in sys_acc
    int sched = 0;                   // traversal launch schedule (0: traverse_group, default shape)

    // stage timing
    struct Mark {
        int stage;
        cudaEvent_t a, b;
    };
    bool prof = false;
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    double prof_ms[8] = {0};
    int64_t prof_calls[8] = {0};
    int64_t launches = 0;
};

namespace {

thread_local char g_create_err[256] = {0};

ff_status create_fail(ff_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_create_err, sizeof(g_create_err), fmt, ap);
    va_end(ap);
    return s;
}

}  // namespace

void ffk::set_thread_error(const char* msg)
{
    std::snprintf(g_create_err, sizeof(g_create_err), "%s", msg);
}

namespace {

ff_status fail(ff_ctx* c, ff_status s, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
        if (s == FF_ECUDA || s == FF_EDEVICE || s == FF_ENONFINITE) c->poisoned = true;
    }
    return s;
}

#define FF_CUDA(ctx, call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), FF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

#define FF_LAUNCHED(ctx)                                                                     \
    do {                                                                                     \
        cudaError_t e_ = cudaGetLastError();                                                 \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), FF_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
    } while (0)

ff_status usable(ff_ctx* c, bool need_particles)
{
    if (!c) return FF_EINVAL;
    if (c->poisoned) return fail(c, FF_ESTATE, "context is poisoned by an earlier error; set particles again");
    if (need_particles && !c->have_particles) return fail(c, FF_ESTATE, "no particles set");
    FF_CUDA(c, cudaSetDevice(c->p.device));
    return FF_OK;
}

size_t dsize(int32_t dtype) { return dtype == FF_DTYPE_F64 ? 8 : 4; }

bool valid_dtype_loc(int32_t dtype, int32_t loc)
{
    return (dtype == FF_DTYPE_F32 || dtype == FF_DTYPE_F64) && (loc == FF_HOST || loc == FF_DEVICE);
}

template <typename R>
ffk::Tree<R> tree_of(ff_ctx* c)
{
    ffk::Tree<R> t;
    t.cell = static_cast<ffk::Cell<R>*>(c->cell);
    t.mom = static_cast<ffk::vec4<R>*>(c->mom);
    t.lo = static_cast<ffk::vec4<R>*>(c->lo);
    t.sum = static_cast<ffk::vec4<R>*>(c->sum);
    t.parent = c->parent;
    t.arrive = c->arrive;
    t.ncells = reinterpret_cast<int*>(c->off + c->n);
    t.cap = c->cap;
    t.q1 = static_cast<ffk::vec4<R>*>(c->q1);
    t.q2 = static_cast<ffk::vec4<R>*>(c->q2);
    // the same cutoff as field_params' rcut (the opening rule's LJ cut)
    const bool lj_on = c->p.lj_eps != 0.0 && c->p.lj_rcut > 0.0;
    t.rcut = lj_on ? (R)c->p.lj_rcut : R(0);
    return t;
}

ffk::Segs segs_of(const ff_ctx* c)
{
    ffk::Segs sg;
    if (c->nsys > 0) {
        sg.of_pos = c->sys_of_pos;
        sg.start = c->sys_start;
        sg.nseg = c->nsys;
    }
    return sg;
}

template <typename R>
ffk::FieldParams<R> field_params(const ff_ctx* c, double theta, int include_sr)
{
    const ff_params& p = c->p;
    ffk::FieldParams<R> fp;
    const bool lj_on = p.lj_eps != 0.0 && p.lj_rcut > 0.0;
    fp.theta2 = (R)(theta * theta);
    fp.rcut2 = lj_on ? (R)(p.lj_rcut * p.lj_rcut) : R(0);
    fp.rcut = lj_on ? (R)p.lj_rcut : R(0);
    fp.use_rcut = lj_on ? 1 : 0;
    fp.include_sr = (include_sr && lj_on) ? 1 : 0;
    fp.dip_scale = (R)p.dip_scale;
    fp.lj_eps24 = (R)(24.0 * p.lj_eps);
    fp.lj_sigma2 = (R)(p.lj_sigma * p.lj_sigma);
    fp.lj_sigma2_lo = (R)(p.lj_sigma * p.lj_sigma - (double)fp.lj_sigma2);
    fp.lj_rcut2 = (R)(p.lj_rcut * p.lj_rcut);
    fp.lj_rcut2_hi = (R)((double)fp.lj_rcut2 * (sizeof(R) == 4 ? 1.0 + 1e-5 : 1.0 + 1e-12));
    const double rin = (p.lj_rcut - 0.01) * (1.0 - 1e-5);
    fp.lj_rcut2_lo = (R)(rin > 0.0 ? rin * rin : 0.0);
    fp.lj_e2 = (R)(2.0 * p.lj_eps);
    fp.lj_e4 = (R)(4.0 * p.lj_eps);
    double sc2 = lj_on ? p.lj_sigma * p.lj_sigma / (p.lj_rcut * p.lj_rcut) : 0.0;
    double sc6 = sc2 * sc2 * sc2;
    fp.lj_shift = (R)(2.0 * p.lj_eps * sc6 * sc6 - 4.0 * p.lj_eps * sc6);
    return fp;
}

template <typename R>
ffk::DynParams<R> dyn_params(const ff_ctx* c)
{
    const ff_params& p = c->p;
    ffk::DynParams<R> d;
    d.dt = (R)p.dt;
    d.gamma_t = (R)p.gamma_t;
    d.gamma_r = (R)p.gamma_r;
    d.inv_inertia = (R)(1.0 / p.inertia);
    d.sig_t = (R)std::sqrt(2.0 * p.gamma_t * p.kT * p.dt);
    d.sig_r = (R)(std::sqrt(p.rot_noise * p.gamma_r * p.kT * p.dt) / p.inertia);
    d.hx = (R)p.h_ext[0];
    d.hy = (R)p.h_ext[1];
    d.hz = (R)p.h_ext[2];
    for (int a = 0; a < 3; ++a) {
        d.lo[a] = (R)(p.box_lo[a] - 0.5);
        d.hi[a] = (R)(p.box_hi[a] + 0.5);
    }
    d.wall_eps24 = (R)(24.0 * p.wall_eps);
    d.wall_e2 = (R)(2.0 * p.wall_eps);
    d.wall_e4 = (R)(4.0 * p.wall_eps);
    d.walls = p.walls ? 1 : 0;
    d.printed_angles = p.rotation == FF_ROT_PRINTED ? 1 : 0;
    d.key0 = (uint32_t)p.seed;
    d.key1 = (uint32_t)(p.seed >> 32);
    d.step = c->dstep;
    d.sys_h = static_cast<const ffk::vec4<R>*>(c->sys_h);
    d.sys_lo = static_cast<const ffk::vec4<R>*>(c->sys_lo);
    d.sys_hi = static_cast<const ffk::vec4<R>*>(c->sys_hi);
    d.sys_of_pos = c->nsys > 0 ? c->sys_of_pos : nullptr;
    d.sys_acc = c->nsys > 0 ? c->sys_acc : nullptr;
    d.flags = c->dflags;
    return d;
}

template <typename R>
ffk::vec4<R>* V(void* p) { return static_cast<ffk::vec4<R>*>(p); }

// Lanes that walk the cell list together (see k_field.cu).
constexpr int kDefaultGroup = 1;
int traverse_group(const ff_ctx* c)
{
    const int g = c->p.traverse_group;
    return (g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32) ? g : kDefaultGroup;
}

enum Stage { S_KEYS = 0, S_SORT, S_GATHER, S_BUILD, S_AGG, S_FIELD, S_STEP, S_OUT };

cudaEvent_t take_event(ff_ctx* c)
{
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one stage with events on the context's stream when timing is on.
struct StageTimer {
    ff_ctx* c;
    int stage;
    cudaEvent_t a = nullptr;
    StageTimer(ff_ctx* cc, int st) : c(cc), stage(st)
    {
        if (c->prof) {
            a = take_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~StageTimer()
    {
        if (!a) return;
        cudaEvent_t b = take_event(c);
        cudaEventRecord(b, c->stream);
        c->marks.push_back({stage, a, b});
    }
};

// Adds the kernels launched during one API call to the context's tally.
struct LaunchTally {
    ff_ctx* c;
    int64_t start;
    explicit LaunchTally(ff_ctx* cc) : c(cc), start(ffk::g_launches.load()) {}
    ~LaunchTally()
    {
        if (c) c->launches += ffk::g_launches.load() - start;
    }
};

// Sort the state into Morton order (the other buffer), build and aggregate
// the tree, traverse.  h, f, esr (and counts) end in sorted order.
template <typename R>
ff_status eval_bh(ff_ctx* c, double theta, int include_sr, bool force_counts = false,
                  const ffk::EntryPool* pool = nullptr, bool field = true)
{
    const int64_t n = c->n;
    cudaStream_t s = c->stream;
    Buffers& a = c->st[c->cur];
    Buffers& b = c->st[1 - c->cur];
    {
        StageTimer st(c, S_KEYS);
        ffk::morton_keys<R>(V<R>(a.pos), n, c->bbox, c->keys[0], c->vals[0], c->dflags,
                            segs_of(c), s);
    }
    {
        StageTimer st(c, S_SORT);
        ffk::radix_sort_pairs(c->keys[0], c->vals[0], c->keys[1], c->vals[1], n, c->radix_tmp,
                              c->dflags, s);
        ffk::radix_sort_systems(c->keys[0], c->vals[0], c->keys[1], c->vals[1], n, c->radix_tmp,
                                segs_of(c), c->dflags, s);
    }
    {
        StageTimer st(c, S_GATHER);
        ffk::gather_state<R>(c->vals[0], n, V<R>(a.pos), V<R>(a.vel), V<R>(a.u), V<R>(a.om), a.id,
                             V<R>(b.pos), V<R>(b.vel), V<R>(b.u), V<R>(b.om), b.id, s);
    }
    c->cur = 1 - c->cur;
    ffk::Tree<R> t = tree_of<R>(c);
    {
        StageTimer st(c, S_BUILD);
        ffk::build_tree<R>(c->keys[0], n, c->p.leaf_max, c->bbox, t, c->cnt, c->off, c->scan_tmp,
                           c->dflags, segs_of(c), s);
    }
    {
        StageTimer st(c, S_AGG);
        if (c->mixed)
            ffk::aggregate_tree<R, double>(V<R>(b.pos), V<R>(b.u), n, c->cnt, c->off, t, c->sum_hi,
                                           c->mom_hi, c->dflags, s);
        else
            ffk::aggregate_tree<R, R>(V<R>(b.pos), V<R>(b.u), n, c->cnt, c->off, t, t.sum, t.mom,
                                      c->dflags, s);
    }
    if (field) {
        StageTimer st(c, S_FIELD);
        if (pool)
            ffk::bh_field_record<R>(V<R>(b.pos), V<R>(b.u), n, t,
                                    field_params<R>(c, theta, include_sr), V<R>(c->h), V<R>(c->f),
                                    static_cast<R*>(c->esr), c->counts, c->dflags, c->work, c->off,
                                    segs_of(c), *pool, s);
        else
            ffk::bh_field<R>(V<R>(b.pos), V<R>(b.u), n, t, field_params<R>(c, theta, include_sr),
                             V<R>(c->h), V<R>(c->f), static_cast<R*>(c->esr),
                             (c->p.count_interactions || force_counts) ? c->counts : nullptr,
                             c->dflags, c->work, traverse_group(c), c->sched, c->off, segs_of(c),
                             s);
    }
    FF_LAUNCHED(c);
    c->tree_valid = true;
    c->counts_valid = field && (c->p.count_interactions != 0 || force_counts || pool);
    return FF_OK;
}

template <typename R>
ff_status eval_ap(ff_ctx* c, int include_sr)
{
    Buffers& a = c->st[c->cur];
    {
        StageTimer st(c, S_FIELD);
        ffk::ap_field<R>(V<R>(a.pos), V<R>(a.u), c->n, field_params<R>(c, 0.0, include_sr),
                         V<R>(c->h), V<R>(c->f), static_cast<R*>(c->esr), c->stream);
    }
    FF_LAUNCHED(c);
    return FF_OK;
}

template <typename R>
ff_status eval_field(ff_ctx* c, int algo, double theta, int include_sr)
{
    return algo == FF_ALGO_AP ? eval_ap<R>(c, include_sr) : eval_bh<R>(c, theta, include_sr);
}

template <typename R>
ff_status do_step(ff_ctx* c)
{
    ff_status st = eval_field<R>(c, c->p.algo, c->p.theta, 1);
    if (st != FF_OK) return st;
    Buffers& a = c->st[c->cur];
    Buffers& b = c->st[1 - c->cur];
    {
        StageTimer tm(c, S_STEP);
        ffk::integrate<R>(c->n, V<R>(a.pos), V<R>(a.vel), V<R>(a.u), V<R>(a.om), a.id, V<R>(c->h),
                          V<R>(c->f), static_cast<R*>(c->esr), dyn_params<R>(c), V<R>(b.pos),
                          V<R>(b.vel), V<R>(b.u), V<R>(b.om), b.id, c->partials, c->stream);
        ffk::reduce_partials(c->partials, ffk::integrate_blocks(c->n), 1.0 / (double)c->n,
                             0.5 * c->p.inertia, c->obs_step, c->stream);
        ffk::step_advance(c->dstep, c->dflags, c->stream);
    }
    FF_LAUNCHED(c);
    c->cur = 1 - c->cur;
    c->step += 1;
    return FF_OK;
}

// Internal status: the cell arrays were grown (and skipped steps run again)
// under the caller, which redoes its work (see retrying).
constexpr ff_status kRetry = static_cast<ff_status>(-100);
ff_status recover_cells(ff_ctx* c);

// Runs body again while it reports that the cells were grown under it.
template <typename F>
ff_status retrying(ff_ctx* c, F&& body)
{
    for (int attempt = 0; attempt < 8; ++attempt) {
        const ff_status s = body();
        if (s != kRetry) return s;
    }
    return fail(c, FF_EDEVICE, "the tree kept outgrowing its cell arrays");
}

// Waits for the stream and turns device flags into a status.
ff_status sync_and_check(ff_ctx* c)
{
    FF_CUDA(c, cudaMemcpyAsync(c->hflags, c->dflags, sizeof(int), cudaMemcpyDeviceToHost,
                               c->stream));
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    const int fl = *c->hflags;
    if (fl & ffk::FLAG_NONFINITE) return fail(c, FF_ENONFINITE, "a particle position is NaN or infinite");
    if (fl & ffk::FLAG_TRAVERSE) return fail(c, FF_EDEVICE, "traversal guard tripped");
    if (fl & ffk::FLAG_AGGREGATE) return fail(c, FF_EDEVICE, "aggregation guard tripped");
    if (fl & ffk::FLAG_SORT) return fail(c, FF_EDEVICE, "a sort or record-scan tile timed out waiting for an earlier tile");
    if (fl & ffk::FLAG_CAPACITY) {
        const ff_status s = recover_cells(c);
        return s == FF_OK ? kRetry : s;
    }
    return FF_OK;
}

void free_all(ff_ctx* c)
{
    void* ptrs[] = {c->keys[0], c->keys[1], c->vals[0], c->vals[1], c->radix_tmp, c->cnt, c->off,
                    c->scan_tmp, c->bbox, c->cell, c->mom, c->lo, c->sum, c->sum_hi, c->mom_hi,
                    c->q1, c->q2, c->parent,
                    c->arrive, c->h, c->f, c->esr, c->counts, c->work, c->partials, c->obs, c->obs_step, c->dstep, c->sys_of_pos, c->sys_start, c->sys_h, c->sys_lo,
                    c->sys_hi, c->sys_acc,
                    c->dflags, c->staging, c->e_cnt, c->e_base, c->e_total, c->g_pos, c->g_u,
                    c->rs_key, c->rs_mask, c->e_tmp, c->s_beg,
                    c->s_end, c->s_G, c->s_Q, c->s_items, c->s_item_off, c->s_scan, c->i_part,
                    c->t_cnt, c->t_off, c->s_rbeg, c->r_key, c->r_idx, c->r_rec, c->r_srec,
                    c->r_E, c->r_scan, c->p_keys, c->p_link, c->p_next, c->s_src};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (int k = 0; k < 2; ++k) {
        void* bp[] = {c->st[k].pos, c->st[k].vel, c->st[k].u, c->st[k].om, c->st[k].id};
        for (void* q : bp)
            if (q) cudaFree(q);
    }
    for (auto& m : c->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k)
        if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
    c->marks.clear();
    c->pool.clear();
    if (c->hflags) cudaFreeHost(c->hflags);
    if (c->hobs) cudaFreeHost(c->hobs);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

template <typename T>
cudaError_t dalloc(T** p, size_t bytes)
{
    return cudaMalloc(reinterpret_cast<void**>(p), bytes > 0 ? bytes : 16);
}

// Cells of the tree.  Every particle starts at most 22 cells (levels 0..21), so
// 22 n + 1 cells always suffice, but gases, chains and dense packings need 1.2
// to 1.8 cells per particle: the arrays start at 2 n + 8192 cells and grow when
// a build needs more (see recover_cells).
int64_t initial_cells(int64_t n)
{
    const int64_t bound = 22 * n + 1;
    const int64_t start = 2 * n + 8192;
    return start < bound ? start : bound;
}

// (Re)allocates every per-cell array for cap cells.
ff_status alloc_cells(ff_ctx* c, int64_t cap)
{
    void* olds[] = {c->cell, c->mom, c->lo, c->sum, c->sum_hi, c->mom_hi, c->q1, c->q2,
                    c->parent, c->arrive};
    for (void* q : olds)
        if (q) cudaFree(q);
    c->cell = c->mom = c->lo = c->sum = c->q1 = c->q2 = nullptr;
    c->sum_hi = c->mom_hi = nullptr;
    c->parent = c->arrive = nullptr;
    c->cap = 0;
    const size_t rec = c->rec;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = dalloc(p, bytes);
    };
    A(&c->cell, c->cell_bytes * cap);
    A(&c->mom, rec * cap);
    A(&c->lo, rec * cap);
    A(&c->sum, rec * cap);
    if (c->mixed) {
        A(&c->sum_hi, sizeof(ffk::dvec4) * cap);
        A(&c->mom_hi, sizeof(ffk::dvec4) * cap);
    }
    if (c->p.quadrupole) {
        A(&c->q1, rec * cap);
        A(&c->q2, rec * cap);
    }
    A(&c->parent, sizeof(int) * cap);
    A(&c->arrive, sizeof(int) * cap);
    if (e != cudaSuccess)
        return fail(c, FF_ENOMEM, "device allocation of %lld cells failed: %s", (long long)cap,
                    cudaGetErrorString(e));
    c->cap = cap;
    c->tree_valid = false;
    c->counts_valid = false;
    return FF_OK;
}

ff_status alloc_all(ff_ctx* c)
{
    const int64_t n = c->n;
    const size_t rec = c->rec;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = dalloc(p, bytes);
    };
    for (int k = 0; k < 2; ++k) {
        A(&c->st[k].pos, rec * n);
        A(&c->st[k].vel, rec * n);
        A(&c->st[k].u, rec * n);
        A(&c->st[k].om, rec * n);
        A(&c->st[k].id, sizeof(uint32_t) * n);
        A(&c->keys[k], sizeof(uint64_t) * n);
        A(&c->vals[k], sizeof(uint32_t) * n);
    }
    A(&c->radix_tmp, sizeof(uint32_t) * ffk::radix_tmp_words(n));
    A(&c->cnt, sizeof(uint32_t) * (n + 1));
    A(&c->off, sizeof(uint32_t) * (n + 1));
    A(&c->scan_tmp, sizeof(uint32_t) * ffk::scan_tmp_words(n));
    A(&c->bbox, sizeof(ffk::BBox));
    A(&c->h, rec * n);
    A(&c->f, rec * n);
    A(&c->esr, (c->fp64 ? 8 : 4) * n);
    A(&c->counts, sizeof(int4) * n);
    A(&c->work, sizeof(int) * ffk::kWorkSegments);
    A(&c->partials, sizeof(double) * ffk::kObs * ffk::integrate_blocks(n));
    A(&c->obs, sizeof(double) * ffk::kObs);
    A(&c->obs_step, sizeof(double) * ffk::kObs);
    A(&c->dstep, sizeof(unsigned long long));
    A(&c->dflags, sizeof(int));
    A(&c->staging, sizeof(double) * 12 * n);
    if (e != cudaSuccess) return fail(c, FF_ENOMEM, "device allocation failed: %s", cudaGetErrorString(e));
    ff_status st = alloc_cells(c, initial_cells(n));
    if (st != FF_OK) return st;
    if (cudaMallocHost(reinterpret_cast<void**>(&c->hflags), sizeof(int)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&c->hobs), sizeof(double) * ffk::kObs) != cudaSuccess)
        return fail(c, FF_ENOMEM, "pinned host allocation failed");
    FF_CUDA(c, cudaMemsetAsync(c->dflags, 0, sizeof(int), c->stream));
    FF_CUDA(c, cudaMemsetAsync(c->obs_step, 0, sizeof(double) * ffk::kObs, c->stream));
    FF_CUDA(c, cudaMemsetAsync(c->dstep, 0, sizeof(unsigned long long), c->stream));
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    return FF_OK;
}

const char* check_params(const ff_params* p)
{
    if (p->struct_size != sizeof(ff_params)) return "struct_size does not match sizeof(ff_params)";
    if (p->n < 1 || p->n > kMaxN) return "n out of range (1 .. 2^27)";
    if (p->precision != FF_FP32 && p->precision != FF_FP64 && p->precision != FF_MIXED)
        return "bad precision";
    if (p->rotation != FF_ROT_VECTOR && p->rotation != FF_ROT_PRINTED) return "bad rotation";
    if (p->quadrupole != 0 && p->quadrupole != 1) return "quadrupole must be 0 or 1";
    if (p->algo != FF_ALGO_BH && p->algo != FF_ALGO_AP) return "bad algo";
    if (p->leaf_max < 1 || p->leaf_max > ffk::kMaxLeaf) return "leaf_max out of range (1 .. 64)";
    if (!(p->theta >= 0.0) || !std::isfinite(p->theta)) return "theta must be finite and >= 0";
    if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return "dt must be > 0";
    if (!(p->inertia > 0.0)) return "inertia must be > 0";
    if (!(p->gamma_t >= 0.0) || !(p->gamma_r >= 0.0)) return "friction must be >= 0";
    if (!(p->kT >= 0.0) || !(p->rot_noise >= 0.0)) return "kT and rot_noise must be >= 0";
    if (!std::isfinite(p->dip_scale)) return "dip_scale must be finite";
    if (p->traverse_group != 0 && p->traverse_group != 1 && p->traverse_group != 2 &&
        p->traverse_group != 4 && p->traverse_group != 8 && p->traverse_group != 16 &&
        p->traverse_group != 32)
        return "traverse_group must be 0, 1, 2, 4, 8, 16 or 32";
    if (p->lj_eps != 0.0 && (!(p->lj_sigma > 0.0) || !(p->lj_rcut > 0.0)))
        return "LJ needs sigma > 0 and rcut > 0";
    if (p->walls) {
        for (int a = 0; a < 3; ++a)
            if (!(p->box_lo[a] < p->box_hi[a])) return "walls need box_lo < box_hi";
        if (!(p->wall_eps >= 0.0)) return "wall_eps must be >= 0";
    }
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->h_ext[a])) return "h_ext must be finite";
    return nullptr;
}

template <typename R>
ff_status load_array(ff_ctx* c, const void* src, int32_t dtype, int32_t loc, void* dst, int slot)
{
    const int64_t n = c->n;
    if (!src) {
        ffk::fill_zero4<R>(V<R>(dst), n, c->stream);
        return FF_OK;
    }
    const void* dsrc = src;
    if (loc == FF_HOST) {
        char* stg = static_cast<char*>(c->staging) + (size_t)slot * 3 * n * sizeof(double);
        FF_CUDA(c, cudaMemcpyAsync(stg, src, 3 * n * dsize(dtype), cudaMemcpyHostToDevice, c->stream));
        dsrc = stg;
    }
    if (dtype == FF_DTYPE_F64)
        ffk::load3<R, double>(static_cast<const double*>(dsrc), n, V<R>(dst), c->stream);
    else
        ffk::load3<R, float>(static_cast<const float*>(dsrc), n, V<R>(dst), c->stream);
    return FF_OK;
}

template <typename R>
ff_status set_particles(ff_ctx* c, const void* pos, const void* u, const void* vel,
                        const void* om, int32_t dtype, int32_t loc)
{
    Buffers& a = c->st[c->cur];
    ff_status s;
    if ((s = load_array<R>(c, pos, dtype, loc, a.pos, 0)) != FF_OK) return s;
    if ((s = load_array<R>(c, u, dtype, loc, a.u, 1)) != FF_OK) return s;
    if ((s = load_array<R>(c, vel, dtype, loc, a.vel, 2)) != FF_OK) return s;
    if ((s = load_array<R>(c, om, dtype, loc, a.om, 3)) != FF_OK) return s;
    ffk::iota32(a.id, c->n, c->stream);
    // a new state: earlier flags no longer apply, and steps that a too small cell array
    // held back are dropped with the state they were for (the noise counter follows
    // the host's step count)
    FF_CUDA(c, cudaMemsetAsync(c->dflags, 0, sizeof(int), c->stream));
    const unsigned long long v = (unsigned long long)c->step;
    FF_CUDA(c, cudaMemcpyAsync(c->dstep, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
    FF_LAUNCHED(c);
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    return FF_OK;
}

// Writes one record array (sorted order) to a caller array in caller order.
template <typename R>
ff_status store_array(ff_ctx* c, const void* src, const uint32_t* id, void* dst, int32_t dtype,
                      int32_t loc, int slot)
{
    if (!dst) return FF_OK;
    const int64_t n = c->n;
    void* ddst = dst;
    char* stg = static_cast<char*>(c->staging) + (size_t)slot * 3 * n * sizeof(double);
    if (loc == FF_HOST) ddst = stg;
    StageTimer tm(c, S_OUT);
    if (dtype == FF_DTYPE_F64)
        ffk::scatter3<R, double>(static_cast<const ffk::vec4<R>*>(src), id, n,
                                 static_cast<double*>(ddst), c->stream);
    else
        ffk::scatter3<R, float>(static_cast<const ffk::vec4<R>*>(src), id, n,
                                static_cast<float*>(ddst), c->stream);
    FF_LAUNCHED(c);
    if (loc == FF_HOST)
        FF_CUDA(c, cudaMemcpyAsync(dst, stg, 3 * n * dsize(dtype), cudaMemcpyDeviceToHost, c->stream));
    return FF_OK;
}

template <typename R>
ff_status get_particles(ff_ctx* c, void* pos, void* u, void* vel, void* om, int32_t dtype,
                        int32_t loc)
{
    Buffers& a = c->st[c->cur];
    ff_status s;
    if ((s = store_array<R>(c, a.pos, a.id, pos, dtype, loc, 0)) != FF_OK) return s;
    if ((s = store_array<R>(c, a.u, a.id, u, dtype, loc, 1)) != FF_OK) return s;
    if ((s = store_array<R>(c, a.vel, a.id, vel, dtype, loc, 2)) != FF_OK) return s;
    if ((s = store_array<R>(c, a.om, a.id, om, dtype, loc, 3)) != FF_OK) return s;
    return sync_and_check(c);
}

template <typename R>
ff_status dipolar_field(ff_ctx* c, int32_t algo, double theta, int32_t include_sr, void* h_out,
                        void* f_out, int32_t dtype, int32_t loc)
{
    ff_status s = eval_field<R>(c, algo, theta, include_sr);
    if (s != FF_OK) return s;
    const uint32_t* id = c->st[c->cur].id;
    if ((s = store_array<R>(c, c->h, id, h_out, dtype, loc, 0)) != FF_OK) return s;
    if ((s = store_array<R>(c, c->f, id, f_out, dtype, loc, 1)) != FF_OK) return s;
    return sync_and_check(c);
}

template <typename R>
ff_status energy(ff_ctx* c, ff_energy_t* out)
{
    ff_status s = eval_field<R>(c, c->p.algo, c->p.theta, 1);
    if (s != FF_OK) return s;
    Buffers& a = c->st[c->cur];
    ffk::observables<R>(c->n, V<R>(a.pos), V<R>(a.vel), V<R>(a.u), V<R>(a.om), V<R>(c->h),
                        static_cast<R*>(c->esr), dyn_params<R>(c), c->partials, c->stream);
    ffk::reduce_partials(c->partials, ffk::integrate_blocks(c->n), 1.0 / (double)c->n,
                         0.5 * c->p.inertia, c->obs, c->stream);
    FF_LAUNCHED(c);
    FF_CUDA(c, cudaMemcpyAsync(c->hobs, c->obs, sizeof(double) * ffk::kObs, cudaMemcpyDeviceToHost,
                               c->stream));
    if ((s = sync_and_check(c)) != FF_OK) return s;
    const double* o = c->hobs;
    out->e_dip = o[0];
    out->e_zeeman = o[1];
    out->e_sr = o[2];
    out->e_wall = o[3];
    out->e_kin_t = o[4];
    out->e_kin_r = o[5];
    out->m[0] = o[6];
    out->m[1] = o[7];
    out->m[2] = o[8];
    out->hdip_z_mean = o[9];
    return FF_OK;
}

// (Re)allocates a device array of count elements; callers track capacity.
template <typename T>
ff_status grow(ff_ctx* c, T** p, size_t count)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(c, FF_ENOMEM, "device allocation for the gradient failed: %s", cudaGetErrorString(e));
    }
    return FF_OK;
}

// After a counted Barnes-Hut evaluation: scans the per-particle interaction
// counts into entry slots and sizes every buffer the recorded entries need.
ff_status prepare_entries(ff_ctx* c, int64_t* ne_out, int64_t* ncells_out, int64_t* max_items_out,
                          int64_t* pool_used)
{
    const int64_t n = c->n;
    cudaStream_t s = c->stream;
    ff_status st;
    if (!c->e_cnt) {
        if ((st = grow(c, &c->e_cnt, n)) != FF_OK) return st;
        if ((st = grow(c, &c->e_base, n + 1)) != FF_OK) return st;
        if ((st = grow(c, &c->e_total, 1)) != FF_OK) return st;
    }
    int ncells_h = 0;
    FF_CUDA(c, cudaMemsetAsync(c->e_total, 0, sizeof(unsigned long long), s));
    ffk::grad_entry_counts(c->counts, n, c->e_cnt, c->e_total, s);
    ffk::scan_exclusive(c->e_cnt, c->e_base, n, c->scan_tmp, s);
    FF_LAUNCHED(c);
    unsigned long long total = 0;
    FF_CUDA(c, cudaMemcpyAsync(&total, c->e_total, sizeof(total), cudaMemcpyDeviceToHost, s));
    FF_CUDA(c, cudaMemcpyAsync(&ncells_h, c->off + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    unsigned taken = 0;
    FF_CUDA(c, cudaMemcpyAsync(&taken, c->p_next, sizeof(taken), cudaMemcpyDeviceToHost, s));
    if ((st = sync_and_check(c)) != FF_OK) return st;
    *pool_used = n + (int64_t)taken;
    // entry positions are 32-bit, with room for the recording walk's 16-byte groups
    if (total >= 0xfffffff0ull)
        return fail(c, FF_EINVAL, "too many interactions (%llu) for one gradient pass", total);
    const int64_t ne = (int64_t)total;
    const int64_t ncells = ncells_h;
    const int64_t nsrc = ncells + n;
    if (ne > c->e_cap) {
        const int64_t cap = ne + ne / 8 + 1024;
        if ((st = grow(c, &c->rs_key, cap)) != FF_OK) return st;
        if ((st = grow(c, &c->rs_mask, cap)) != FF_OK) return st;
        if ((st = grow(c, &c->e_tmp, ffk::radix_tmp_words(cap))) != FF_OK) return st;
        c->e_cap = cap;
    }
    if (nsrc > c->s_cap) {
        const int64_t cap = nsrc + nsrc / 8 + 1024;
        if ((st = grow(c, &c->s_beg, cap)) != FF_OK) return st;
        if ((st = grow(c, &c->s_end, cap)) != FF_OK) return st;
        if ((st = grow(c, &c->s_G, 3 * cap)) != FF_OK) return st;
        if ((st = grow(c, &c->s_Q, 3 * cap)) != FF_OK) return st;
        if ((st = grow(c, &c->s_items, cap)) != FF_OK) return st;
        if ((st = grow(c, &c->s_item_off, cap + 1)) != FF_OK) return st;
        if ((st = grow(c, &c->s_scan, ffk::scan_tmp_words(cap))) != FF_OK) return st;
        if ((st = grow(c, &c->s_rbeg, cap)) != FF_OK) return st;
        if ((st = grow(c, &c->s_src, cap)) != FF_OK) return st;
        c->s_cap = cap;
    }
    const int64_t max_items = nsrc + ne / ffk::kGradItemEntries + 1;
    if (max_items > c->i_cap) {
        const int64_t cap = max_items + max_items / 8 + 1024;
        // six partial sums per item, then the item -> source map (half a double each)
        if ((st = grow(c, &c->i_part, 7 * cap)) != FF_OK) return st;
        c->i_cap = cap;
    }
    *ne_out = ne;
    *ncells_out = ncells;
    *max_items_out = max_items;
    return FF_OK;
}

// The entry pool of the recording walk: at least `chunks` chunks.
ff_status grow_pool(ff_ctx* c, int64_t chunks)
{
    ff_status st;
    if (chunks <= c->p_cap) return FF_OK;
    if (chunks > 0xffffffffll)
        return fail(c, FF_EINVAL, "too many interactions (%lld chunks) for one gradient pass",
                    (long long)chunks);
    if ((st = grow(c, &c->p_keys, (size_t)chunks * ffk::kPoolChunk)) != FF_OK) return st;
    if ((st = grow(c, &c->p_link, chunks)) != FF_OK) return st;
    if (!c->p_next && (st = grow(c, &c->p_next, 1)) != FF_OK) return st;
    c->p_cap = chunks;
    return FF_OK;
}

ffk::EntryPool pool_of(ff_ctx* c)
{
    ffk::EntryPool p;
    p.keys = c->p_keys;
    p.link = c->p_link;
    p.next = c->p_next;
    p.cap = (uint32_t)c->p_cap;
    p.first = (uint32_t)c->n;
    return p;
}

// The pool ready for a recording walk: room for at least n + 1024 chunks (9 per
// particle at first), its counter cleared.
ff_status pool_prepare(ff_ctx* c)
{
    ff_status st;
    if (c->p_cap < c->n + 1024 && (st = grow_pool(c, 9 * c->n + 1024)) != FF_OK) return st;
    FF_CUDA(c, cudaMemsetAsync(c->p_next, 0, sizeof(unsigned), c->stream));
    return FF_OK;
}

// After the recording walk and prepare_entries (which read the chunks it took):
// a pool that ran out is grown to what the walk took and the walk redone (the
// same field, force, counts and lists).
template <typename R>
ff_status pool_settle(ff_ctx* c, double theta, int include_sr, int64_t used)
{
    if (used <= c->p_cap) return FF_OK;
    ff_status st;
    if ((st = grow_pool(c, used + used / 8 + 1024)) != FF_OK) return st;
    FF_CUDA(c, cudaMemsetAsync(c->p_next, 0, sizeof(unsigned), c->stream));
    Buffers& a = c->st[c->cur];
    ffk::bh_field_record<R>(V<R>(a.pos), V<R>(a.u), c->n, tree_of<R>(c),
                            field_params<R>(c, theta, include_sr), V<R>(c->h), V<R>(c->f),
                            static_cast<R*>(c->esr), c->counts, c->dflags, c->work, c->off,
                            segs_of(c), pool_of(c), c->stream);
    FF_LAUNCHED(c);
    return FF_OK;
}

// After the recording walk and prepare_entries: each task's sources gathered into
// records, packed, sorted by their place in the depth-first order and scanned
// into entry offsets (k_grad.cu).  Waits to read the number of records.
template <typename R>
ff_status record_sources(ff_ctx* c, int64_t ncells, int64_t* nrec_out)
{
    const int64_t n = c->n;
    const int64_t nsrc = ncells + n;
    const int64_t ntask = (n + 31) / 32;
    cudaStream_t s = c->stream;
    ff_status st;
    if (!c->t_cnt) {
        if ((st = grow(c, &c->t_cnt, ntask)) != FF_OK) return st;
        if ((st = grow(c, &c->t_off, ntask + 1)) != FF_OK) return st;
    }
    // the records of task T go to the slots of its particles (rs_key, rs_mask)
    ffk::grad_merge_records(c->e_cnt, n, pool_of(c), c->e_base, c->rs_key, c->rs_mask,
                            c->t_cnt, c->dflags, s);
    ffk::scan_exclusive(c->t_cnt, c->t_off, ntask, c->scan_tmp, s);
    ffk::grad_source_map<R>(tree_of<R>(c), ncells, c->s_src, s);
    FF_LAUNCHED(c);
    uint32_t total = 0;
    FF_CUDA(c, cudaMemcpyAsync(&total, c->t_off + ntask, sizeof(total), cudaMemcpyDeviceToHost, s));
    if ((st = sync_and_check(c)) != FF_OK) return st;
    const int64_t nrec = total;
    if (nrec > c->r_cap) {
        const int64_t cap = nrec + nrec / 8 + 1024;
        if ((st = grow(c, &c->r_key, cap)) != FF_OK) return st;
        if ((st = grow(c, &c->r_idx, cap)) != FF_OK) return st;
        if ((st = grow(c, &c->r_rec, cap)) != FF_OK) return st;
        if ((st = grow(c, &c->r_srec, cap)) != FF_OK) return st;
        if ((st = grow(c, &c->r_E, cap + 1)) != FF_OK) return st;
        if ((st = grow(c, &c->r_scan, ffk::record_scan_words(cap))) != FF_OK) return st;
        c->r_cap = cap;
    }
    ffk::grad_pack_records(c->t_cnt, c->t_off, ntask, c->e_base, c->rs_key, c->rs_mask,
                           c->r_key, c->r_idx, c->r_rec, s);
    int passes = 1;
    while (passes < 4 && ((uint64_t)nsrc >> (8 * passes)) != 0) ++passes;
    // the records, in task order, sorted stably by source (rs_key, rs_mask
    // are free again and serve as the other buffer pair)
    const bool in1 = ffk::radix_sort_pairs_passes<uint32_t>(
        c->r_key, c->r_idx, c->rs_key, c->rs_mask, nrec, c->e_tmp, passes, c->dflags, s);
    const uint32_t* skey = in1 ? c->rs_key : c->r_key;
    const uint32_t* sidx = in1 ? c->rs_mask : c->r_idx;
    ffk::grad_record_sources(skey, sidx, nrec, c->r_rec, c->s_src, nsrc, c->r_srec, c->r_E,
                             c->r_scan, c->s_rbeg, c->s_beg, c->s_end, c->dflags, s);
    FF_LAUNCHED(c);
    *nrec_out = nrec;
    return FF_OK;
}

// Energy -1/2 sum u.h (FP64) and its gradient with the opening decisions of
// this evaluation frozen (k_grad.cu), in sorted order in g_pos, g_u.
template <typename R>
ff_status energy_grad(ff_ctx* c, int32_t algo, double theta, double* energy, bool grads)
{
    const int64_t n = c->n;
    cudaStream_t s = c->stream;
    ff_status st;
    if (!grads) {
        // the energy alone: one field evaluation and the FP64 reduction
        if ((st = eval_field<R>(c, algo, theta, 0)) != FF_OK) return st;
    } else if (!c->g_pos) {
        if ((st = grow(c, reinterpret_cast<char**>(&c->g_pos), c->rec * n)) != FF_OK) return st;
        if ((st = grow(c, reinterpret_cast<char**>(&c->g_u), c->rec * n)) != FF_OK) return st;
    }
    if (!grads) {
    } else if (algo == FF_ALGO_AP) {
        if ((st = eval_ap<R>(c, 0)) != FF_OK) return st;
        ffk::grad_from_field<R>(V<R>(c->h), V<R>(c->f), n, V<R>(c->g_pos), V<R>(c->g_u), s);
        FF_LAUNCHED(c);
    } else {
        // the field, the counts and every particle's sources in one walk
        if ((st = pool_prepare(c)) != FF_OK) return st;
        const ffk::EntryPool pool = pool_of(c);
        if ((st = eval_bh<R>(c, theta, 0, true, &pool)) != FF_OK) return st;
        int64_t ne = 0, ncells = 0, max_items = 0, used = 0;
        if ((st = prepare_entries(c, &ne, &ncells, &max_items, &used)) != FF_OK) return st;
        if ((st = pool_settle<R>(c, theta, 0, used)) != FF_OK) return st;
        Buffers& a = c->st[c->cur];
        ffk::Tree<R> t = tree_of<R>(c);
        int64_t nrec = 0;
        if ((st = record_sources<R>(c, ncells, &nrec)) != FF_OK) return st;
        ffk::grad_source_sums_rec<R>(V<R>(a.pos), V<R>(a.u), t, ncells, n, c->r_srec, c->r_E,
                                     nrec, c->s_rbeg, c->s_beg, c->s_end, c->s_items,
                                     c->s_item_off, c->s_scan, c->i_part, max_items, c->s_G,
                                     c->s_Q, s);
        ffk::grad_finish<R>(t, ncells, n, c->s_G, c->s_Q, V<R>(c->h), V<R>(c->f),
                            (R)c->p.dip_scale, V<R>(c->g_pos), V<R>(c->g_u), s);
        FF_LAUNCHED(c);
    }
    Buffers& a = c->st[c->cur];
    ffk::observables<R>(n, V<R>(a.pos), V<R>(a.vel), V<R>(a.u), V<R>(a.om), V<R>(c->h),
                        static_cast<R*>(c->esr), dyn_params<R>(c), c->partials, s);
    ffk::reduce_partials(c->partials, ffk::integrate_blocks(n), 1.0 / (double)n,
                         0.5 * c->p.inertia, c->obs, s);
    FF_LAUNCHED(c);
    FF_CUDA(c, cudaMemcpyAsync(c->hobs, c->obs, sizeof(double) * ffk::kObs, cudaMemcpyDeviceToHost,
                               s));
    if ((st = sync_and_check(c)) != FF_OK) return st;
    if (energy) *energy = c->hobs[0];
    return FF_OK;
}

}  // namespace

namespace {

// Sorts and builds once, then times the traversal for each candidate: lane group
// groups[i] with launch schedule scheds[i] (scheds may be null: the default shape).
template <typename R>
ff_status tune_traversal(ff_ctx* c, const int32_t* groups, const int32_t* scheds, int ng, int reps,
                         float* ms_out, int* best)
{
    ff_status s = eval_bh<R>(c, c->p.theta, 1);
    if (s != FF_OK) return s;
    if ((s = sync_and_check(c)) != FF_OK) return s;
    Buffers& a = c->st[c->cur];
    ffk::Tree<R> t = tree_of<R>(c);
    const ffk::FieldParams<R> fp = field_params<R>(c, c->p.theta, 1);
    struct Events {
        std::vector<cudaEvent_t> v;
        ~Events()
        {
            for (cudaEvent_t e : v)
                if (e) cudaEventDestroy(e);
        }
    } hold;
    hold.v.assign(2 * (size_t)ng * reps, nullptr);
    std::vector<cudaEvent_t>& ev = hold.v;
    for (auto& e : ev) FF_CUDA(c, cudaEventCreate(&e));
    for (int g = 0; g < ng; ++g)
        for (int r = 0; r < reps; ++r) {
            cudaEvent_t* e = &ev[2 * ((size_t)g * reps + r)];
            cudaEventRecord(e[0], c->stream);
            ffk::bh_field<R>(V<R>(a.pos), V<R>(a.u), c->n, t, fp, V<R>(c->h), V<R>(c->f),
                             static_cast<R*>(c->esr), nullptr, c->dflags, c->work, groups[g],
                             scheds ? scheds[g] : 0, c->off, segs_of(c), c->stream);
            cudaEventRecord(e[1], c->stream);
        }
    FF_LAUNCHED(c);
    s = sync_and_check(c);
    float best_ms = 0.0f;
    *best = 0;
    for (int g = 0; g < ng && s == FF_OK; ++g) {
        float m = 0.0f;
        for (int r = 0; r < reps; ++r) {
            float x = 0.0f;
            cudaEventElapsedTime(&x, ev[2 * ((size_t)g * reps + r)], ev[2 * ((size_t)g * reps + r) + 1]);
            m = (r == 0 || x < m) ? x : m;
        }
        if (ms_out) ms_out[g] = m;
        if (g == 0 || m < best_ms) {
            best_ms = m;
            *best = g;
        }
    }
    return s;
}

// Sensitivity of the mean magnetisation over nsteps steps to the applied
// field, by reverse mode through every step (k_step.cu em_adjoint, the field
// and force VJP of k_field.cu / k_grad.cu), with the state saved every
// `every` steps and each segment recomputed on the way back.
template <typename R>
ff_status mz_sensitivity(ff_ctx* c, int64_t nsteps, int64_t every, double* mz_out, double* g_out)
{
    const int64_t n = c->n;
    cudaStream_t s = c->stream;
    const size_t rb = c->rec * (size_t)n;
    const size_t ib = sizeof(uint32_t) * (size_t)n;
    const int64_t ncp = (nsteps + every - 1) / every;
    struct Scratch {
        std::vector<void*> dev;
        double* host = nullptr;
        ~Scratch()
        {
            for (void* q : dev) cudaFree(q);
            if (host) cudaFreeHost(host);
        }
    } sc;
    bool oom = false;
    auto alloc = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes ? bytes : 1) != cudaSuccess) {
            oom = true;
            return nullptr;
        }
        sc.dev.push_back(q);
        return q;
    };
    struct Snap {
        void* a[4];
        uint32_t* id;
        int64_t step;
    };
    auto new_snap = [&](Snap& d) {
        for (int q = 0; q < 4; ++q) d.a[q] = alloc(rb);
        d.id = static_cast<uint32_t*>(alloc(ib));
        d.step = 0;
    };
    std::vector<Snap> cps((size_t)ncp), seg((size_t)(every < nsteps ? every : nsteps));
    Snap fin;
    for (auto& d : cps) new_snap(d);
    for (auto& d : seg) new_snap(d);
    new_snap(fin);
    // the field of each recomputed step (its particles' sorted order), for its adjoint
    std::vector<void*> hseg(seg.size());
    for (auto& q : hseg) q = alloc(rb);
    R* adj[4];
    R* tmp[4];
    for (int q = 0; q < 4; ++q) {
        adj[q] = static_cast<R*>(alloc(rb));
        tmp[q] = static_cast<R*>(alloc(rb));
    }
    R* abar = static_cast<R*>(alloc(rb));
    R* bbar = static_cast<R*>(alloc(rb));
    R* dxt = static_cast<R*>(alloc(rb));
    R* dut = static_cast<R*>(alloc(rb));
    const int nb = ffk::integrate_blocks(n);
    double* hpart = static_cast<double*>(alloc(sizeof(double) * 3 * nb));
    double* mzs = static_cast<double*>(alloc(sizeof(double) * nsteps));
    double* sumtmp = static_cast<double*>(alloc(sizeof(double) * ffk::sum_tmp_words(n)));
    if (oom) return fail(c, FF_ENOMEM, "device allocation for the sensitivity failed");
    if (cudaMallocHost(reinterpret_cast<void**>(&sc.host), sizeof(double) * (3 * nb + nsteps)) !=
        cudaSuccess)
        return fail(c, FF_ENOMEM, "pinned host allocation for the sensitivity failed");
    double* hp_host = sc.host;
    double* mz_host = sc.host + 3 * nb;

    auto save = [&](Snap& d) -> ff_status {
        Buffers& b = c->st[c->cur];
        void* src[4] = {b.pos, b.vel, b.u, b.om};
        for (int q = 0; q < 4; ++q)
            FF_CUDA(c, cudaMemcpyAsync(d.a[q], src[q], rb, cudaMemcpyDeviceToDevice, s));
        FF_CUDA(c, cudaMemcpyAsync(d.id, b.id, ib, cudaMemcpyDeviceToDevice, s));
        d.step = c->step;
        return FF_OK;
    };
    auto load = [&](const Snap& d) -> ff_status {
        Buffers& b = c->st[c->cur];
        void* dst[4] = {b.pos, b.vel, b.u, b.om};
        for (int q = 0; q < 4; ++q)
            FF_CUDA(c, cudaMemcpyAsync(dst[q], d.a[q], rb, cudaMemcpyDeviceToDevice, s));
        FF_CUDA(c, cudaMemcpyAsync(b.id, d.id, ib, cudaMemcpyDeviceToDevice, s));
        c->step = d.step;
        ffk::step_set(c->dstep, (unsigned long long)d.step, s);
        return FF_OK;
    };

    // forward, saving the state every `every` steps; M_z of every new state
    ff_status st;
    for (int64_t t = 0; t < nsteps; ++t) {
        if (t % every == 0 && (st = save(cps[(size_t)(t / every)])) != FF_OK) return st;
        if ((st = do_step<R>(c)) != FF_OK) return st;
        ffk::sum_z<R>(V<R>(c->st[c->cur].u), n, sumtmp, mzs + t, s);
        FF_LAUNCHED(c);
    }
    if ((st = save(fin)) != FF_OK) return st;
    FF_CUDA(c, cudaMemcpyAsync(mz_host, mzs, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, s));
    if ((st = sync_and_check(c)) != FF_OK) return st;
    double mz = 0.0;
    for (int64_t t = 0; t < nsteps; ++t) mz += mz_host[t];
    mz /= (double)n * (double)nsteps;

    // backward, one segment at a time from the last
    for (int q = 0; q < 4; ++q) FF_CUDA(c, cudaMemsetAsync(adj[q], 0, rb, s));
    double hsum[3] = {0.0, 0.0, 0.0};
    const R add_uz = (R)(1.0 / ((double)n * (double)nsteps));
    const double theta = c->p.theta;
    for (int64_t cp = ncp - 1; cp >= 0; --cp) {
        const int64_t t0 = cp * every, t1 = std::min(nsteps, t0 + every);
        if ((st = load(cps[(size_t)cp])) != FF_OK) return st;
        for (int64_t t = t0; t < t1; ++t) {
            if ((st = save(seg[(size_t)(t - t0)])) != FF_OK) return st;
            if ((st = do_step<R>(c)) != FF_OK) return st;
            FF_CUDA(c, cudaMemcpyAsync(hseg[(size_t)(t - t0)], c->h, rb, cudaMemcpyDeviceToDevice,
                                       s));
        }
        for (int64_t t = t1 - 1; t >= t0; --t) {
            if ((st = load(seg[(size_t)(t - t0)])) != FF_OK) return st;
            // the step's tree and decisions (the state is sorted), its field as the
            // recomputed step left it, the cotangents of the field and force, then one
            // walk for the target-side terms that also writes the source lists
            if ((st = eval_bh<R>(c, theta, 1, false, nullptr, false)) != FF_OK) return st;
            FF_CUDA(c, cudaMemcpyAsync(c->h, hseg[(size_t)(t - t0)], rb, cudaMemcpyDeviceToDevice,
                                       s));
            Buffers& a = c->st[c->cur];
            const uint32_t* perm = c->vals[0];
            ffk::em_adjoint<R>(n, V<R>(a.pos), V<R>(a.u), V<R>(a.om), V<R>(c->h), dyn_params<R>(c),
                               add_uz, V<R>(adj[0]), V<R>(adj[1]), V<R>(adj[2]), V<R>(adj[3]),
                               V<R>(abar), V<R>(bbar), hpart, s);
            FF_LAUNCHED(c);
            FF_CUDA(c, cudaMemcpyAsync(hp_host, hpart, sizeof(double) * 3 * nb,
                                       cudaMemcpyDeviceToHost, s));
            ffk::Tree<R> tr = tree_of<R>(c);
            auto vjp_walk = [&]() -> ff_status {
                const ffk::EntryPool pool = pool_of(c);
                ffk::bh_vjp_target<R>(V<R>(a.pos), V<R>(a.u), V<R>(abar), V<R>(bbar), n, tr,
                                      field_params<R>(c, theta, 1), c->dflags, c->work, c->off,
                                      segs_of(c), V<R>(dxt), V<R>(dut), s, c->counts, &pool);
                FF_LAUNCHED(c);
                return FF_OK;
            };
            if ((st = pool_prepare(c)) != FF_OK) return st;
            if ((st = vjp_walk()) != FF_OK) return st;
            int64_t ne = 0, ncells = 0, max_items = 0, used = 0;
            if ((st = prepare_entries(c, &ne, &ncells, &max_items, &used)) != FF_OK) return st;
            for (int b = 0; b < nb; ++b)
                for (int q = 0; q < 3; ++q) hsum[q] += hp_host[3 * b + q];
            if (used > c->p_cap) {
                // a pool that ran out: grown to what the walk took, the walk redone
                if ((st = grow_pool(c, used + used / 8 + 1024)) != FF_OK) return st;
                FF_CUDA(c, cudaMemsetAsync(c->p_next, 0, sizeof(unsigned), s));
                if ((st = vjp_walk()) != FF_OK) return st;
            }
            c->counts_valid = false;  // entries per particle, not the counting walk's split
            int64_t nrec = 0;
            if ((st = record_sources<R>(c, ncells, &nrec)) != FF_OK) return st;
            ffk::vjp_source_sums_rec<R>(V<R>(a.pos), V<R>(a.u), V<R>(abar), V<R>(bbar),
                                        (R)c->p.dip_scale, tr, ncells, n, c->r_srec, c->r_E, nrec,
                                        c->s_rbeg, c->s_beg, c->s_end, c->s_items, c->s_item_off,
                                        c->s_scan, c->i_part, max_items, c->s_G, c->s_Q, s);
            ffk::vjp_finish<R>(tr, ncells, n, c->s_G, c->s_Q, V<R>(dxt), V<R>(dut), V<R>(adj[0]),
                               V<R>(adj[2]), s);
            // carry the adjoints back through the step's gather into the state's order
            for (int q = 0; q < 4; ++q) {
                ffk::scatter_records<R>(perm, n, V<R>(adj[q]), V<R>(tmp[q]), s);
                std::swap(adj[q], tmp[q]);
            }
            FF_LAUNCHED(c);
        }
    }
    if ((st = load(fin)) != FF_OK) return st;
    if ((st = sync_and_check(c)) != FF_OK) return st;
    if (mz_out) *mz_out = mz;
    if (g_out)
        for (int q = 0; q < 3; ++q) g_out[q] = hsum[q];
    return FF_OK;
}

}  // namespace

// =================================================================== C ABI
namespace {

template <typename R>
void fill_sys_records(std::vector<unsigned char>& out, int nsys, const double* v3, double add,
                      const double* fallback)
{
    out.assign(sizeof(ffk::vec4<R>) * nsys, 0);
    ffk::vec4<R>* r = reinterpret_cast<ffk::vec4<R>*>(out.data());
    for (int s = 0; s < nsys; ++s) {
        const double* src = v3 ? v3 + 3 * (size_t)s : fallback;
        r[s].x = (R)(src[0] + add);
        r[s].y = (R)(src[1] + add);
        r[s].z = (R)(src[2] + add);
        r[s].w = R(0);
    }
}

void drop_graphs(ff_ctx* c)
{
    for (int k = 0; k < 2; ++k)
        if (c->gexec[k]) {
            cudaGraphExecDestroy(c->gexec[k]);
            c->gexec[k] = nullptr;
        }
}

}  // namespace

extern "C" {

void ff_params_default(ff_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->struct_size = sizeof(ff_params);
    p->precision = FF_FP32;
    p->n = 1;
    p->algo = FF_ALGO_BH;
    p->leaf_max = 1;
    p->theta = 0.5;
    p->dt = 1e-3;
    p->gamma_t = 0.1;
    p->gamma_r = 0.1;
    p->inertia = 0.4;
    p->kT = 1.0;
    p->rot_noise = 2.0;
    p->dip_scale = 1.0;
    p->lj_eps = 1.0;
    p->lj_sigma = 1.0;
    p->lj_rcut = 2.5;
    p->walls = 0;
    p->device = 0;
    p->wall_eps = 1.0;
    p->seed = 1;
    p->count_interactions = 0;
    p->stream = nullptr;
}

ff_status ff_create(const ff_params* p, ff_ctx** out)
{
    if (!p || !out) return create_fail(FF_EINVAL, "p and out must not be NULL");
    *out = nullptr;
    if (const char* why = check_params(p)) return create_fail(FF_EINVAL, "%s", why);
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return create_fail(FF_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    ff_ctx* c = new (std::nothrow) ff_ctx();
    if (!c) return create_fail(FF_ENOMEM, "host allocation failed");
    c->p = *p;
    c->n = p->n;
    c->fp64 = p->precision == FF_FP64;
    c->mixed = p->precision == FF_MIXED;
    c->rec = c->fp64 ? sizeof(ffk::dvec4) : sizeof(float4);
    c->cell_bytes = c->fp64 ? sizeof(ffk::Cell<double>) : sizeof(ffk::Cell<float>);
    if (p->stream) {
        c->stream = static_cast<cudaStream_t>(p->stream);
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return create_fail(FF_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    ff_status s = alloc_all(c);
    if (s != FF_OK) {
        create_fail(s, "%s", c->err);
        free_all(c);
        delete c;
        return s;
    }
    g_create_err[0] = 0;
    *out = c;
    return FF_OK;
}

ff_status ff_destroy(ff_ctx* c)
{
    if (!c) return FF_OK;
    cudaSetDevice(c->p.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return FF_OK;
}

ff_status ff_set_particles(ff_ctx* c, const void* pos, const void* u, const void* vel,
                           const void* omega, int32_t dtype, int32_t loc)
{
    LaunchTally tally_(c);
    if (!c) return FF_EINVAL;
    if (!pos || !u) return fail(c, FF_EINVAL, "pos and u are required");
    if (!valid_dtype_loc(dtype, loc)) return fail(c, FF_EINVAL, "bad dtype or loc");
    FF_CUDA(c, cudaSetDevice(c->p.device));
    c->poisoned = false;
    c->cur = 0;
    ff_status s = c->fp64 ? set_particles<double>(c, pos, u, vel, omega, dtype, loc)
                          : set_particles<float>(c, pos, u, vel, omega, dtype, loc);
    if (s != FF_OK) return s;
    c->have_particles = true;
    c->tree_valid = false;
    c->counts_valid = false;
    return FF_OK;
}

ff_status ff_get_particles(ff_ctx* c, void* pos, void* u, void* vel, void* omega, int32_t dtype,
                           int32_t loc)
{
    LaunchTally tally_(c);
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    if (!valid_dtype_loc(dtype, loc)) return fail(c, FF_EINVAL, "bad dtype or loc");
    return retrying(c, [&] {
        return c->fp64 ? get_particles<double>(c, pos, u, vel, omega, dtype, loc)
                       : get_particles<float>(c, pos, u, vel, omega, dtype, loc);
    });
}

ff_status ff_dipolar_field(ff_ctx* c, int32_t algo, double theta, int32_t include_sr, void* h_out,
                           void* f_out, int32_t dtype, int32_t loc)
{
    LaunchTally tally_(c);
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    if (algo != FF_ALGO_BH && algo != FF_ALGO_AP) return fail(c, FF_EINVAL, "bad algo");
    if (algo == FF_ALGO_AP && c->nsys > 0) return fail(c, FF_EINVAL, "all-pairs is not available for batched systems");
    if (!(theta >= 0.0) || !std::isfinite(theta)) return fail(c, FF_EINVAL, "theta must be finite and >= 0");
    if (!valid_dtype_loc(dtype, loc)) return fail(c, FF_EINVAL, "bad dtype or loc");
    return retrying(c, [&] {
        return c->fp64 ? dipolar_field<double>(c, algo, theta, include_sr, h_out, f_out, dtype, loc)
                       : dipolar_field<float>(c, algo, theta, include_sr, h_out, f_out, dtype, loc);
    });
}

ff_status ff_energy_grad(ff_ctx* c, int32_t algo, double theta, double* energy, void* grad_pos,
                         void* grad_u, int32_t dtype, int32_t loc)
{
    LaunchTally tally_(c);
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    if (algo != FF_ALGO_BH && algo != FF_ALGO_AP) return fail(c, FF_EINVAL, "bad algo");
    if (algo == FF_ALGO_AP && c->nsys > 0) return fail(c, FF_EINVAL, "all-pairs is not available for batched systems");
    if (!(theta >= 0.0) || !std::isfinite(theta)) return fail(c, FF_EINVAL, "theta must be finite and >= 0");
    if (!valid_dtype_loc(dtype, loc)) return fail(c, FF_EINVAL, "bad dtype or loc");
    if (c->p.quadrupole && algo == FF_ALGO_BH)
        return fail(c, FF_EINVAL, "the gradient uses the paper's pseudo-particles (quadrupole off)");
    const bool grads = grad_pos != nullptr || grad_u != nullptr;
    return retrying(c, [&] {
        ff_status st = c->fp64 ? energy_grad<double>(c, algo, theta, energy, grads)
                               : energy_grad<float>(c, algo, theta, energy, grads);
        if (st != FF_OK || !grads) return st;
        const uint32_t* id = c->st[c->cur].id;
        if (c->fp64) {
            if ((st = store_array<double>(c, c->g_pos, id, grad_pos, dtype, loc, 0)) != FF_OK) return st;
            if ((st = store_array<double>(c, c->g_u, id, grad_u, dtype, loc, 1)) != FF_OK) return st;
        } else {
            if ((st = store_array<float>(c, c->g_pos, id, grad_pos, dtype, loc, 0)) != FF_OK) return st;
            if ((st = store_array<float>(c, c->g_u, id, grad_u, dtype, loc, 1)) != FF_OK) return st;
        }
        return sync_and_check(c);
    });
}

ff_status ff_mz_sensitivity(ff_ctx* c, int64_t nsteps, int64_t every, double* mz, double* dmz_dh)
{
    LaunchTally tally_(c);
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    if (c->p.rotation != FF_ROT_VECTOR) return fail(c, FF_EINVAL, "the sensitivity is defined for the vector rotor");
    if (c->p.quadrupole) return fail(c, FF_EINVAL, "the sensitivity uses the paper's pseudo-particles (quadrupole off)");
    if (nsteps < 1) return fail(c, FF_EINVAL, "nsteps must be >= 1");
    if (every < 1) return fail(c, FF_EINVAL, "every must be >= 1");
    if (c->nsys > 0) return fail(c, FF_EINVAL, "the sensitivity is for a single system");
    if (c->p.algo != FF_ALGO_BH) return fail(c, FF_EINVAL, "the context does not use Barnes-Hut");
    // steps issued before this call are complete (and their trees fitted) first
    if ((s = retrying(c, [&] { return sync_and_check(c); })) != FF_OK) return s;
    s = c->fp64 ? mz_sensitivity<double>(c, nsteps, every, mz, dmz_dh)
                : mz_sensitivity<float>(c, nsteps, every, mz, dmz_dh);
    if (s == kRetry)
        return fail(c, FF_EDEVICE, "a tree outgrew the cell arrays during the run; they have been "
                                   "grown, set the state again and repeat the call");
    return s;
}

}  // extern "C"

namespace {

// nsteps steps, each one captured CUDA graph launch (eager launches while stage
// timing is on); asynchronous.
ff_status run_steps(ff_ctx* c, int64_t nsteps)
{
    ff_status s = FF_OK;
    if (c->prof) {
        // stage timing needs the events between stages: launch eagerly
        for (int64_t k = 0; k < nsteps; ++k) {
            s = c->fp64 ? do_step<double>(c) : do_step<float>(c);
            if (s != FF_OK) return s;
            if (c->nsys > 0) c->sys_steps += 1;
        }
        return FF_OK;
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        const int start = c->cur;
        if (!c->gexec[start]) {
            // capture one step; nothing runs during capture, so the buffer index
            // and the host step counter are put back afterwards
            const int64_t l0 = ffk::g_launches.load();
            const int64_t step0 = c->step;
            FF_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            s = c->fp64 ? do_step<double>(c) : do_step<float>(c);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
            if (s != FF_OK) {
                if (graph) cudaGraphDestroy(graph);
                return s;
            }
            if (e != cudaSuccess) return fail(c, FF_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&c->gexec[start], graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail(c, FF_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
            c->gend[start] = c->cur;
            c->glaunch[start] = ffk::g_launches.load() - l0;
            ffk::g_launches.fetch_sub(c->glaunch[start]);
            c->cur = start;
            c->step = step0;
        }
        FF_CUDA(c, cudaGraphLaunch(c->gexec[start], c->stream));
        ffk::counted((int)c->glaunch[start]);
        c->cur = c->gend[start];
        c->step += 1;
        if (c->nsys > 0) c->sys_steps += 1;
        c->tree_valid = c->tree_valid || c->p.algo == FF_ALGO_BH;
        c->counts_valid = c->p.algo == FF_ALGO_BH && c->p.count_interactions != 0;
    }
    return FF_OK;
}

// A build needed more cells than allocated (FLAG_CAPACITY): that step and every
// step after it left the state and the step counter unchanged.  Grows the cell
// arrays to 1.25 x what the current state needs, clears the flag and runs again
// the steps that were issued since.  The caller then redoes its own work.
ff_status recover_cells(ff_ctx* c)
{
    uint32_t need = 0;
    unsigned long long dstep = 0;
    FF_CUDA(c, cudaMemcpy(&need, c->off + c->n, sizeof(need), cudaMemcpyDeviceToHost));
    FF_CUDA(c, cudaMemcpy(&dstep, c->dstep, sizeof(dstep), cudaMemcpyDeviceToHost));
    const int64_t bound = 22 * c->n + 1;
    int64_t want = (int64_t)need + (int64_t)need / 4 + 8192;
    if (want <= c->cap) want = 2 * c->cap;
    if (want > bound) want = bound;
    drop_graphs(c);  // the captured steps use the old arrays
    ff_status s = alloc_cells(c, want);
    if (s != FF_OK) return s;
    FF_CUDA(c, cudaMemsetAsync(c->dflags, 0, sizeof(int), c->stream));
    const int64_t missing = c->step - (int64_t)dstep;
    if (missing > 0) {
        c->step = (int64_t)dstep;
        if (c->nsys > 0) c->sys_steps -= missing;
        if ((s = run_steps(c, missing)) != FF_OK) return s;
    }
    return FF_OK;
}

}  // namespace

extern "C" {

ff_status ff_step(ff_ctx* c, int64_t nsteps)
{
    LaunchTally tally_(c);
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    if (nsteps < 0) return fail(c, FF_EINVAL, "nsteps must be >= 0");
    if (c->p.algo == FF_ALGO_AP && c->nsys > 0) return fail(c, FF_EINVAL, "all-pairs is not available for batched systems");
    return run_steps(c, nsteps);
}

ff_status ff_energy(ff_ctx* c, ff_energy_t* out)
{
    LaunchTally tally_(c);
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    if (!out) return fail(c, FF_EINVAL, "out is NULL");
    if (c->p.algo == FF_ALGO_AP && c->nsys > 0) return fail(c, FF_EINVAL, "all-pairs is not available for batched systems");
    return retrying(c, [&] { return c->fp64 ? energy<double>(c, out) : energy<float>(c, out); });
}

ff_status ff_get_step(const ff_ctx* c, int64_t* step)
{
    if (!c || !step) return FF_EINVAL;
    *step = c->step;
    return FF_OK;
}

ff_status ff_set_step(ff_ctx* c, int64_t step)
{
    if (!c) return FF_EINVAL;
    if (step < 0) return fail(c, FF_EINVAL, "step must be >= 0");
    FF_CUDA(c, cudaSetDevice(c->p.device));
    const unsigned long long v = (unsigned long long)step;
    FF_CUDA(c, cudaMemcpyAsync(c->dstep, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    c->step = step;
    return FF_OK;
}

ff_status ff_synchronize(ff_ctx* c)
{
    ff_status s = usable(c, false);
    if (s != FF_OK) return s;
    return retrying(c, [&] { return sync_and_check(c); });
}

ff_status ff_tree_info(ff_ctx* c, ff_tree_info_t* out)
{
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    if (!out) return fail(c, FF_EINVAL, "out is NULL");
    if (!c->tree_valid) return fail(c, FF_ESTATE, "no Barnes-Hut tree has been built");
    if ((s = retrying(c, [&] { return sync_and_check(c); })) != FF_OK) return s;
    std::memset(out, 0, sizeof(*out));
    uint32_t nc = 0;
    FF_CUDA(c, cudaMemcpy(&nc, c->off + c->n, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    out->ncells = nc;
    std::vector<int4> nodes(nc);
    if (nc) FF_CUDA(c, cudaMemcpy2D(nodes.data(), sizeof(int4), c->cell, c->cell_bytes, sizeof(int4), nc, cudaMemcpyDeviceToHost));
    int depth = 0;
    for (const int4& v : nodes) depth = std::max(depth, v.w & 0xff);
    out->depth = depth;
    ffk::BBox bb;
    FF_CUDA(c, cudaMemcpy(&bb, c->bbox, sizeof(bb), cudaMemcpyDeviceToHost));
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        if (c->fp64) {
            long long e0 = bb.lo[a], e1 = bb.hi[a];
            e0 = e0 >= 0 ? e0 : e0 ^ 0x7fffffffffffffffLL;
            e1 = e1 >= 0 ? e1 : e1 ^ 0x7fffffffffffffffLL;
            std::memcpy(&mn[a], &e0, 8);
            std::memcpy(&mx[a], &e1, 8);
        } else {
            int e0 = (int)bb.lo[a], e1 = (int)bb.hi[a];
            e0 = e0 >= 0 ? e0 : e0 ^ 0x7fffffff;
            e1 = e1 >= 0 ? e1 : e1 ^ 0x7fffffff;
            float f0, f1;
            std::memcpy(&f0, &e0, 4);
            std::memcpy(&f1, &e1, 4);
            mn[a] = f0;
            mx[a] = f1;
        }
    }
    double side = 0.0;
    if (c->fp64) {
        side = mx[0] - mn[0];
        for (int a = 1; a < 3; ++a) side = std::max(side, mx[a] - mn[a]);
        if (!(side > 0.0)) side = 1.0;
    } else {
        float sd = (float)mx[0] - (float)mn[0];
        for (int a = 1; a < 3; ++a) sd = std::max(sd, (float)mx[a] - (float)mn[a]);
        if (!(sd > 0.0f)) sd = 1.0f;
        side = sd;
    }
    for (int a = 0; a < 3; ++a) out->root[a] = mn[a];
    out->root[3] = side;
    if (c->counts_valid) {
        std::vector<int4> cn(c->n);
        FF_CUDA(c, cudaMemcpy(cn.data(), c->counts, sizeof(int4) * c->n, cudaMemcpyDeviceToHost));
        for (const int4& v : cn) {
            out->accepted += v.x;
            out->pairs += v.y;
            out->opened += v.z;
        }
        out->interactions = out->accepted + out->pairs;
    }
    return FF_OK;
}

ff_status ff_get_tree(ff_ctx* c, uint64_t* keys, uint32_t* order, int32_t* pbegin, int32_t* pend,
                      int32_t* skip, int32_t* level, int32_t* leaf, void* centre, void* moment,
                      int32_t dtype)
{
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    if (!c->tree_valid) return fail(c, FF_ESTATE, "no Barnes-Hut tree has been built");
    if (dtype != FF_DTYPE_F32 && dtype != FF_DTYPE_F64) return fail(c, FF_EINVAL, "bad dtype");
    if ((s = retrying(c, [&] { return sync_and_check(c); })) != FF_OK) return s;
    const int64_t n = c->n;
    uint32_t nc = 0;
    FF_CUDA(c, cudaMemcpy(&nc, c->off + n, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (keys) FF_CUDA(c, cudaMemcpy(keys, c->keys[0], sizeof(uint64_t) * n, cudaMemcpyDeviceToHost));
    if (order) FF_CUDA(c, cudaMemcpy(order, c->st[c->cur].id, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    if (pbegin || pend || skip || level || leaf) {
        std::vector<int4> nodes(nc);
        if (nc) FF_CUDA(c, cudaMemcpy2D(nodes.data(), sizeof(int4), c->cell, c->cell_bytes, sizeof(int4), nc, cudaMemcpyDeviceToHost));
        for (uint32_t i = 0; i < nc; ++i) {
            if (pbegin) pbegin[i] = nodes[i].x;
            if (pend) pend[i] = nodes[i].y;
            if (skip) skip[i] = nodes[i].z;
            if (level) level[i] = nodes[i].w & 0xff;
            if (leaf) leaf[i] = (nodes[i].w >> 8) & 1;
        }
    }
    // the centre is the second half of each Cell record; the moment sum is its own array
    void* srcs[2] = {static_cast<char*>(c->cell) + (c->fp64 ? offsetof(ffk::Cell<double>, cen) : offsetof(ffk::Cell<float>, cen)), c->mom};
    const size_t pitch[2] = {c->cell_bytes, c->rec};
    void* dsts[2] = {centre, moment};
    for (int q = 0; q < 2; ++q) {
        if (!dsts[q] || nc == 0) continue;
        std::vector<unsigned char> raw((size_t)nc * c->rec);
        FF_CUDA(c, cudaMemcpy2D(raw.data(), c->rec, srcs[q], pitch[q], c->rec, nc, cudaMemcpyDeviceToHost));
        for (uint32_t i = 0; i < nc; ++i) {
            double v[3];
            if (c->fp64) {
                const double* r = reinterpret_cast<const double*>(raw.data() + (size_t)i * c->rec);
                v[0] = r[0]; v[1] = r[1]; v[2] = r[2];
            } else {
                const float* r = reinterpret_cast<const float*>(raw.data() + (size_t)i * c->rec);
                v[0] = r[0]; v[1] = r[1]; v[2] = r[2];
            }
            for (int a = 0; a < 3; ++a) {
                if (dtype == FF_DTYPE_F64) static_cast<double*>(dsts[q])[3 * (size_t)i + a] = v[a];
                else static_cast<float*>(dsts[q])[3 * (size_t)i + a] = (float)v[a];
            }
        }
    }
    return FF_OK;
}

ff_status ff_get_counts(ff_ctx* c, int32_t* accepted, int32_t* pairs, int32_t* opened)
{
    LaunchTally tally_(c);
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    if (!c->counts_valid) return fail(c, FF_ESTATE, "no interaction counts recorded (count_interactions = 0 or no BH evaluation)");
    const int64_t n = c->n;
    int32_t* stg = static_cast<int32_t*>(c->staging);
    ffk::scatter_counts<float>(c->counts, c->st[c->cur].id, n, stg, stg + n, stg + 2 * n, c->stream);
    FF_LAUNCHED(c);
    if ((s = retrying(c, [&] { return sync_and_check(c); })) != FF_OK) return s;
    int32_t* dst[3] = {accepted, pairs, opened};
    for (int q = 0; q < 3; ++q)
        if (dst[q]) FF_CUDA(c, cudaMemcpy(dst[q], stg + q * n, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    return FF_OK;
}

ff_status ff_set_systems(ff_ctx* c, int32_t nsys, const int64_t* counts, const double* h_ext,
                         const double* box_lo, const double* box_hi)
{
    if (!c) return FF_EINVAL;
    if (nsys < 1 || nsys > 65536 || !counts) return fail(c, FF_EINVAL, "nsys must be 1 .. 65536 with counts");
    int64_t total = 0;
    for (int s = 0; s < nsys; ++s) {
        if (counts[s] < 1) return fail(c, FF_EINVAL, "every system needs at least one particle");
        total += counts[s];
    }
    if (total != c->n) return fail(c, FF_EINVAL, "system counts must add up to n");
    if (c->p.walls && box_lo && box_hi)
        for (int s = 0; s < nsys; ++s)
            for (int a = 0; a < 3; ++a)
                if (!(box_lo[3 * s + a] < box_hi[3 * s + a])) return fail(c, FF_EINVAL, "walls need box_lo < box_hi");
    FF_CUDA(c, cudaSetDevice(c->p.device));
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    drop_graphs(c);
    void* olds[] = {c->sys_of_pos, c->sys_start, c->sys_h, c->sys_lo, c->sys_hi, c->sys_acc, c->bbox};
    for (void* q : olds)
        if (q) cudaFree(q);
    c->sys_of_pos = nullptr;
    c->sys_start = nullptr;
    c->sys_h = c->sys_lo = c->sys_hi = nullptr;
    c->sys_acc = nullptr;
    c->bbox = nullptr;
    c->nsys = 0;
    std::vector<int> start(nsys + 1, 0);
    std::vector<uint32_t> of_pos(c->n);
    for (int s = 0; s < nsys; ++s) {
        start[s + 1] = start[s] + (int)counts[s];
        for (int64_t i = start[s]; i < start[s + 1]; ++i) of_pos[i] = (uint32_t)s;
    }
    std::vector<unsigned char> rh, rlo, rhi;
    const double* blo = box_lo;
    const double* bhi = box_hi;
    if (c->fp64) {
        fill_sys_records<double>(rh, nsys, h_ext, 0.0, c->p.h_ext);
        fill_sys_records<double>(rlo, nsys, blo, -0.5, c->p.box_lo);
        fill_sys_records<double>(rhi, nsys, bhi, 0.5, c->p.box_hi);
    } else {
        fill_sys_records<float>(rh, nsys, h_ext, 0.0, c->p.h_ext);
        fill_sys_records<float>(rlo, nsys, blo, -0.5, c->p.box_lo);
        fill_sys_records<float>(rhi, nsys, bhi, 0.5, c->p.box_hi);
    }
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = dalloc(p, bytes);
    };
    A(&c->sys_of_pos, sizeof(uint32_t) * c->n);
    A(&c->sys_start, sizeof(int) * (nsys + 1));
    A(&c->sys_h, rh.size());
    A(&c->sys_lo, rlo.size());
    A(&c->sys_hi, rhi.size());
    A(&c->sys_acc, sizeof(double) * 4 * nsys);
    A(&c->bbox, sizeof(ffk::BBox) * nsys);
    if (e != cudaSuccess) return fail(c, FF_ENOMEM, "device allocation failed: %s", cudaGetErrorString(e));
    FF_CUDA(c, cudaMemcpy(c->sys_of_pos, of_pos.data(), sizeof(uint32_t) * c->n, cudaMemcpyHostToDevice));
    FF_CUDA(c, cudaMemcpy(c->sys_start, start.data(), sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice));
    FF_CUDA(c, cudaMemcpy(c->sys_h, rh.data(), rh.size(), cudaMemcpyHostToDevice));
    FF_CUDA(c, cudaMemcpy(c->sys_lo, rlo.data(), rlo.size(), cudaMemcpyHostToDevice));
    FF_CUDA(c, cudaMemcpy(c->sys_hi, rhi.data(), rhi.size(), cudaMemcpyHostToDevice));
    FF_CUDA(c, cudaMemset(c->sys_acc, 0, sizeof(double) * 4 * nsys));
    c->nsys = nsys;
    c->sys_steps = 0;
    c->tree_valid = false;
    c->counts_valid = false;
    return FF_OK;
}

ff_status ff_tune_traversal(ff_ctx* c, const int32_t* groups, int32_t ngroups, int32_t reps,
                            int32_t* best_group, float* ms)
{
    LaunchTally tally_(c);
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    static const int32_t all[6] = {1, 2, 4, 8, 16, 32};
    if (!best_group) return fail(c, FF_EINVAL, "best_group is required");
    if (!groups) {
        if (ngroups != 0) return fail(c, FF_EINVAL, "groups = NULL needs ngroups = 0");
        groups = all;
        ngroups = 6;
    }
    if (ngroups < 1 || ngroups > 64) return fail(c, FF_EINVAL, "ngroups must be 1 .. 64");
    for (int g = 0; g < ngroups; ++g) {
        const int32_t v = groups[g];
        if (v != 1 && v != 2 && v != 4 && v != 8 && v != 16 && v != 32)
            return fail(c, FF_EINVAL, "every candidate must be 1, 2, 4, 8, 16 or 32");
    }
    if (reps < 1 || reps > 100) return fail(c, FF_EINVAL, "reps must be 1 .. 100");
    if (c->p.algo != FF_ALGO_BH) return fail(c, FF_EINVAL, "the context does not use Barnes-Hut");
    int best = 0;
    const int sched0 = c->sched;
    c->sched = 0;  // a group choice replaces a tuned launch schedule
    s = retrying(c, [&] {
        return c->fp64 ? tune_traversal<double>(c, groups, nullptr, ngroups, reps, ms, &best)
                       : tune_traversal<float>(c, groups, nullptr, ngroups, reps, ms, &best);
    });
    if (s != FF_OK) {
        c->sched = sched0;
        return s;
    }
    if (c->p.traverse_group != groups[best] || sched0 != 0) {
        c->p.traverse_group = groups[best];
        drop_graphs(c);  // the captured step launches the old schedule
    }
    *best_group = groups[best];
    return FF_OK;
}

int32_t ff_schedule_count(void) { return ffk::kNumSchedules; }

ff_status ff_schedule_info(int32_t index, int32_t* group, int32_t* threads, int32_t* blocks_per_sm)
{
    if (index < 1 || index > ffk::kNumSchedules) return FF_EINVAL;
    const ffk::Schedule& q = ffk::kSchedules[index - 1];
    if (group) *group = q.group;
    if (threads) *threads = q.threads;
    if (blocks_per_sm) *blocks_per_sm = q.blocks_per_sm;
    return FF_OK;
}

ff_status ff_set_schedule(ff_ctx* c, int32_t index)
{
    if (!c) return FF_EINVAL;
    if (index < 0 || index > ffk::kNumSchedules)
        return fail(c, FF_EINVAL, "schedule must be 0 .. %d", ffk::kNumSchedules);
    if (c->sched != index) {
        c->sched = index;
        drop_graphs(c);
    }
    return FF_OK;
}

ff_status ff_tune_schedule(ff_ctx* c, int32_t reps, int32_t* best_schedule, float* ms)
{
    LaunchTally tally_(c);
    ff_status s = usable(c, true);
    if (s != FF_OK) return s;
    if (!best_schedule) return fail(c, FF_EINVAL, "best_schedule is required");
    if (reps < 1 || reps > 100) return fail(c, FF_EINVAL, "reps must be 1 .. 100");
    if (c->p.algo != FF_ALGO_BH) return fail(c, FF_EINVAL, "the context does not use Barnes-Hut");
    int32_t groups[ffk::kNumSchedules], scheds[ffk::kNumSchedules];
    for (int i = 0; i < ffk::kNumSchedules; ++i) {
        groups[i] = ffk::kSchedules[i].group;
        scheds[i] = i + 1;
    }
    int best = 0;
    s = retrying(c, [&] {
        return c->fp64 ? tune_traversal<double>(c, groups, scheds, ffk::kNumSchedules, reps, ms, &best)
                       : tune_traversal<float>(c, groups, scheds, ffk::kNumSchedules, reps, ms, &best);
    });
    if (s != FF_OK) return s;
    if (c->sched != best + 1) {
        c->sched = best + 1;
        drop_graphs(c);
    }
    *best_schedule = best + 1;
    return FF_OK;
}

ff_status ff_system_moments(ff_ctx* c, double* out, int64_t* nsteps, int32_t reset)
{
    ff_status s = usable(c, false);
    if (s != FF_OK) return s;
    if (c->nsys < 1) return fail(c, FF_ESTATE, "no systems set (ff_set_systems)");
    if ((s = retrying(c, [&] { return sync_and_check(c); })) != FF_OK) return s;
    if (out) FF_CUDA(c, cudaMemcpy(out, c->sys_acc, sizeof(double) * 4 * c->nsys, cudaMemcpyDeviceToHost));
    if (nsteps) *nsteps = c->sys_steps;
    if (reset) {
        FF_CUDA(c, cudaMemset(c->sys_acc, 0, sizeof(double) * 4 * c->nsys));
        c->sys_steps = 0;
    }
    return FF_OK;
}

ff_status ff_profile(ff_ctx* c, int32_t enable)
{
    if (!c) return FF_EINVAL;
    FF_CUDA(c, cudaSetDevice(c->p.device));
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto& m : c->marks) {
        c->pool.push_back(m.a);
        c->pool.push_back(m.b);
    }
    c->marks.clear();
    if (enable) {
        for (int i = 0; i < 8; ++i) {
            c->prof_ms[i] = 0.0;
            c->prof_calls[i] = 0;
        }
        c->launches = 0;
    }
    c->prof = enable != 0;
    return FF_OK;
}

ff_status ff_profile_read(ff_ctx* c, ff_profile_t* out)
{
    if (!c || !out) return FF_EINVAL;
    FF_CUDA(c, cudaSetDevice(c->p.device));
    FF_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto& m : c->marks) {
        float ms = 0.0f;
        FF_CUDA(c, cudaEventElapsedTime(&ms, m.a, m.b));
        c->prof_ms[m.stage] += ms;
        c->prof_calls[m.stage] += 1;
        c->pool.push_back(m.a);
        c->pool.push_back(m.b);
    }
    c->marks.clear();
    for (int i = 0; i < 8; ++i) {
        out->ms[i] = c->prof_ms[i];
        out->calls[i] = c->prof_calls[i];
    }
    out->launches = c->launches;
    return FF_OK;
}

const char* ff_last_error(const ff_ctx* c)
{
    if (!c) return g_create_err;
    return c->err;
}

const char* ff_status_string(ff_status s)
{
    switch (s) {
        case FF_OK: return "FF_OK";
        case FF_EINVAL: return "FF_EINVAL";
        case FF_ENOMEM: return "FF_ENOMEM";
        case FF_ECUDA: return "FF_ECUDA";
        case FF_EDEVICE: return "FF_EDEVICE";
        case FF_ENONFINITE: return "FF_ENONFINITE";
        case FF_ESTATE: return "FF_ESTATE";
    }
    return "unknown status";
}

}  // extern "C"
