// Internal declarations shared by the CUDA translation units of libff.
// Kernels are templated on the arithmetic type R (float or double); every
// launcher takes the stream explicitly and enqueues asynchronously.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace ffk {

// Sets the message returned by ff_last_error(NULL) on the calling thread.
void set_thread_error(const char* msg);

// Kernels launched by this library (all contexts); read as differences.
extern std::atomic<int64_t> g_launches;
inline void counted(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// 32-byte aligned 4-vector of doubles (one 32-byte load per record).
struct alignas(32) dvec4 {
    double x, y, z, w;
};

template <typename R> struct V4;
template <> struct V4<float> { using T = float4; };
template <> struct V4<double> { using T = dvec4; };
template <typename R> using vec4 = typename V4<R>::T;

// Device error flags (one int32 word per context).
enum : int {
    FLAG_NONFINITE = 1,   // a position was NaN or infinite
    FLAG_TRAVERSE = 2,    // traversal guard tripped (corrupt skip pointers)
    FLAG_CAPACITY = 4,    // more cells than allocated
    FLAG_AGGREGATE = 8,   // aggregation walk exceeded the level bound
    FLAG_SORT = 16,       // a sort (or record-scan) tile waited too long for an earlier tile's counts
};

constexpr int kMaxLevel = 21;        // 21 bits per axis -> 63-bit Morton keys
constexpr int kMaxLeaf = 64;         // largest leaf_max accepted
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;

// One-sweep radix sort (one scatter launch per pass, tiles chained by
// decoupled look-back): tile shape and scratch.  The scratch holds the digit
// counts of every pass, then two status arrays of one 64-bit word per tile and
// digit (alternate passes use alternate arrays; each tile clears its words in
// the other array for the pass after it), then one tile ticket per pass.
constexpr int kOsThreads = 256;  // = kRadixBins: one digit per thread
constexpr int kOsItems = 16;     // keys per thread per tile
constexpr int kOsTile = kOsThreads * kOsItems;  // the smallest tile (sizes the scratch)
// Large tiles carry many bytes per look-back and per block-wide scan, and
// keep the look-back chains of a pass short (all tiles of a 1M-key pass run
// at once).  The tile is staged in dynamic shared memory.
// 32-bit keys (the gradient's entries, hundreds of millions) take twice as
// many per thread: 8192-key tiles in the same shared memory.
template <typename K>
constexpr int os_items() { return sizeof(K) == 4 ? 2 * kOsItems : kOsItems; }
template <typename K>
constexpr int os_min_blocks() { return 2; }
template <typename K>
constexpr size_t os_dyn_smem()
{
    return (size_t)kOsThreads * os_items<K>() * (sizeof(K) + sizeof(uint32_t));
}
constexpr int kOsMaxPasses = 8;
constexpr int64_t os_tiles(int64_t n) { return (n + kOsTile - 1) / kOsTile; }
constexpr size_t os_tmp_words(int64_t n)
{
    return (size_t)kOsMaxPasses * kRadixBins + 4 * (size_t)kRadixBins * (size_t)os_tiles(n) +
           kOsMaxPasses;
}

// Root cube, written by the bbox kernels and read by the key kernel.
// lo/hi hold order-preserving integer encodings of the extrema.
struct BBox {
    long long lo[3];
    long long hi[3];
};

// Independent systems advanced together (batched ensembles).  System s owns
// the fixed positions [start[s], start[s+1]) of the particle order at all
// times (keys are sorted within each system), has its own root cube, tree,
// applied field and box.  A single system is described by null pointers.
struct Segs {
    const uint32_t* of_pos = nullptr;  // system of each position (n entries)
    const int* start = nullptr;        // nseg + 1 position offsets
    int nseg = 1;
};

// Field evaluation parameters in the arithmetic type.
template <typename R>
struct FieldParams {
    R theta2;        // theta^2 rounded to R once from the double product
    R rcut2;         // opening-test cut: lj_rcut^2 (0 when LJ is off)
    R rcut;          // lj_rcut (0 when LJ is off)
    R dip_scale;
    R lj_eps24;      // 24 eps
    R lj_sigma2;     // sigma^2 rounded to R
    R lj_sigma2_lo;  // sigma^2 - lj_sigma2 (the FP32 pair's low part; 0 in FP64)
    R lj_rcut2;      // rcut^2: the pair cut (decided on an exactly rounded r^2)
    R lj_rcut2_hi;   // slightly above lj_rcut2: pre-test on a fused r^2
    R lj_rcut2_lo;   // ((rcut - 0.01)(1 - 1e-5))^2: a particle this close is surely
                     // within rcut of its own cell's cube
    R lj_e2, lj_e4;  // 2 eps, 4 eps (pair energy)
    R lj_shift;      // pair energy at rcut
    int use_rcut;    // LJ on: cells closer than rcut are always opened
    int include_sr;  // add the LJ force to f
};

// Integrator parameters (Sec. 2 reduced equations; Sec. 4 Euler-Maruyama).
template <typename R>
struct DynParams {
    R dt, gamma_t, gamma_r, inv_inertia, sig_t, sig_r;
    R hx, hy, hz;
    R lo[3], hi[3];
    R wall_eps24, wall_e2, wall_e4;
    int walls;
    int printed_angles;                  // 1: the printed angle equations (see k_step.cu)
    uint32_t key0, key1;                 // Philox key (seed)
    const unsigned long long* step;      // device word: the step counter
    // batched ensembles (null for a single system): per-system applied field
    // and wall planes, system of each position, per-system sums of u and h_dip_z
    const vec4<R>* sys_h;                // nseg records: h_ext xyz
    const vec4<R>* sys_lo;               // nseg records: box_lo - 1/2
    const vec4<R>* sys_hi;               // nseg records: box_hi + 1/2
    const uint32_t* sys_of_pos;
    double* sys_acc;                     // nseg x 4 (u_x, u_y, u_z, h_dip_z), accumulated
    // the context's error flags (null: none): a step taken while FLAG_CAPACITY is
    // raised (its tree did not fit) leaves the state unchanged
    const int* flags;
};

// What the traversal reads for every visited cell, in one record (32 bytes
// in single precision): topology and the pseudo-particle position.
template <typename R>
struct alignas(32) Cell {
    int4 node;     // pbegin, pend, skip, level | leaf << 8 | (one-particle leaf) << 9
    vec4<R> cen;   // geometric centre xyz, cube side squared (rounded once)
};

// Tree arrays (device pointers), cells in depth-first preorder.
template <typename R>
struct Tree {
    Cell<R>* cell;       // topology + centre
    vec4<R>* mom;        // moment sum xyz; w = far2 of the LJ opening test (see k_field.cu)
    vec4<R>* lo;         // lower cube corner xyz, cube side
    vec4<R>* sum;        // position sum xyz (aggregation scratch)
    int* parent;         // parent cell (-1 for the root)
    int* arrive;         // aggregation arrival counters
    int* ncells;         // device word: number of cells
    int64_t cap;         // allocated cells
    // dipole-position (quadrupole) terms about the centre, when enabled (else null):
    // q1 = (S_xx, S_yy, S_zz, S_xy), q2 = (S_xz, S_yz, m, 0), S the symmetric part of
    // sum (rho_i - c) (x) u_i and m its trace
    vec4<R>* q1 = nullptr;
    vec4<R>* q2 = nullptr;
    R rcut = R(0);       // LJ cutoff of the opening rule (0: LJ off)
};

// Square of the distance from a cell's centre beyond which a particle is
// surely at least rcut from the cell's cube: (rcut + reach) with a margin far
// above the rounding of the distance, of the centre and of reach, where
// reach bounds the distance from the centre to any point of the cube.
template <typename R>
__host__ __device__ __forceinline__ R far2_of(R rcut, R reach)
{
    const R far = (rcut + reach) * R(1.00001) + R(0.01);
    return far * far;
}

// ---------------------------------------------------------------- launchers
// Scan: exclusive prefix sum of n uint32 values into out[0..n]; out[n] = total.
// tmp must hold scan_tmp_words(n) words.
size_t scan_tmp_words(int64_t n);
void scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs, keys < 2^63, eight passes of
// eight bits: the sorted data end in (k0, v0); (k1, v1) is scratch.  tmp must
// hold radix_tmp_words(n) words, 8-byte aligned.  A tile that gives up waiting
// for an earlier tile raises FLAG_SORT in flags (the order is then undefined).
size_t radix_tmp_words(int64_t n);
void radix_sort_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n,
                      uint32_t* tmp, int* flags, cudaStream_t s);
// The same on the low 8 * passes bits only (K = uint64_t or uint32_t keys,
// passes 1 .. 8); returns true when the sorted data ended in (k1, v1) (an odd
// number of passes).
template <typename K>
bool radix_sort_pairs_passes(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int64_t n, uint32_t* tmp,
                             int passes, int* flags, cudaStream_t s);

// One pass of the 64-bit key sort in which tile 0 withholds its digit counts
// and every look-back word is polled once: the bounded wait of tile 1 runs out
// and raises FLAG_SORT.  The keys are then misplaced (every write stays inside
// [0, n)); only the self-test calls it, and nothing reads its output.
void radix_sort_wait_selftest(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n,
                              uint32_t* tmp, int* flags, cudaStream_t s);

// bb holds one root cube per system.
template <typename R>
void morton_keys(const vec4<R>* pos, int64_t n, BBox* bb, uint64_t* keys, uint32_t* vals,
                 int* flags, Segs sg, cudaStream_t s);

// Stable passes on the system of each element (the element's value is its
// position before the sort), restoring system-major order after the key passes.
void radix_sort_systems(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n,
                        uint32_t* tmp, Segs sg, int* flags, cudaStream_t s);

template <typename R>
void gather_state(const uint32_t* perm, int64_t n, const vec4<R>* pos, const vec4<R>* vel,
                  const vec4<R>* u, const vec4<R>* om, const uint32_t* id, vec4<R>* pos2,
                  vec4<R>* vel2, vec4<R>* u2, vec4<R>* om2, uint32_t* id2, cudaStream_t s);

// Tree build from sorted keys: cnt/off are n+1 words of scratch.
template <typename R>
void build_tree(const uint64_t* skeys, int64_t n, int leaf_max, const BBox* bb, Tree<R> t,
                uint32_t* cnt, uint32_t* off, uint32_t* scan_tmp, int* flags, Segs sg,
                cudaStream_t s);

// Aggregation sums in A (R, or double for single-precision trees whose cell
// sums are formed in FP64); ssum/smom hold the A sums (the tree's own sum and
// mom arrays when A = R).
template <typename R, typename A>
void aggregate_tree(const vec4<R>* pos, const vec4<R>* u, int64_t n, const uint32_t* cnt,
                    const uint32_t* off, Tree<R> t, vec4<A>* ssum, vec4<A>* smom, int* flags,
                    cudaStream_t s);

// Target-side terms of a vector-Jacobian product of h and f with cotangents
// abar, bbar (see k_field.cu), on the traversal's decisions: each particle's
// dL/dx and dL/du from its own sources, to dxt, dut.  With a pool (declared
// below) the same walk also writes every particle's sources there and their
// number to counts[k].x (counts[k].y = 0).
struct EntryPool;
template <typename R>
void bh_vjp_target(const vec4<R>* pos, const vec4<R>* u, const vec4<R>* abar, const vec4<R>* bbar,
                   int64_t n, Tree<R> t, FieldParams<R> fp, int* flags, int* work,
                   const uint32_t* off, Segs sg, vec4<R>* dxt, vec4<R>* dut, cudaStream_t s,
                   int4* counts = nullptr, const EntryPool* pool = nullptr);

// Source lists written by the counting traversal of the gradient pass: the
// sources of particle k, in the order of its walk, fill chunk k of kPoolChunk
// keys and then chunks first + 0, first + 1, .. in the order *next (zeroed
// before the walk) hands them out; link[c] is the chunk after c.  A source is
// named by its place in the depth-first order of cells and particles (cell c:
// c + first particle of c; particle p of leaf L: L + 1 + p), so each list
// rises strictly.  Chunks at or past cap are not written: first + *next then
// ends above cap and the walk must be redone with more chunks.
constexpr int kPoolChunk = 128;
struct EntryPool {
    uint32_t* keys = nullptr;  // cap x kPoolChunk
    uint32_t* link = nullptr;  // cap
    unsigned* next = nullptr;
    uint32_t cap = 0;
    uint32_t first = 0;        // the first chunk handed out (n)
};
// bh_field of the one-lane walk with counts, also writing every particle's
// sources to the pool.
template <typename R>
void bh_field_record(const vec4<R>* pos, const vec4<R>* u, int64_t n, Tree<R> t, FieldParams<R> fp,
                     vec4<R>* h, vec4<R>* f, R* esr, int4* counts, int* flags, int* work,
                     const uint32_t* off, Segs sg, EntryPool pool, cudaStream_t s);

// ------------------------------------------------ energy gradient (k_grad.cu)
// entries per particle (accepted cells + exact pairs) as uint32; *total64
// (zeroed by the caller) receives their sum in 64 bits
void grad_entry_counts(const int4* counts, int64_t n, uint32_t* out,
                       unsigned long long* total64, cudaStream_t s);
// The records of every task of 32 particles from their source lists (cnt[k]
// sources of particle k in the pool): each source some particle of the task has
// is written once, with the mask of the lanes that have it, to rkeys/rmask from
// base[32 task] on (base: scan of cnt), and the task's number of records to
// tcount[task].  A block per task collects them in a shared-memory hash table
// (in no particular order); a task with too many sources for it is merged by
// one warp from its rising lists instead (in rising order).
void grad_merge_records(const uint32_t* cnt, int64_t n, EntryPool pool, const uint32_t* base,
                        uint32_t* rkeys, uint32_t* rmask, uint32_t* tcount, int* flags,
                        cudaStream_t s);
// The source named by each place of the depth-first order (cells: the cell,
// particles of multi-particle leaves: ncells + the particle): src_of[ncells + n].
template <typename R>
void grad_source_map(Tree<R> t, int64_t ncells, uint32_t* src_of, cudaStream_t s);
// Records packed in task order: the ntask tasks' records (tcount each, from
// base[32 task] in rkeys/rmask; toff = exclusive scan of tcount) to ckey (the
// key), cidx[r] = r, crec[r] = (task, lane mask).
void grad_pack_records(const uint32_t* tcount, const uint32_t* toff, int64_t ntask,
                       const uint32_t* base, const uint32_t* rkeys, const uint32_t* rmask,
                       uint32_t* ckey, uint32_t* cidx, uint2* crec, cudaStream_t s);
// After the records are sorted by key (skey, sidx = their packed index):
// srec[i] = crec[sidx[i]], recE[i] = entries before record i (recE[nrec] =
// entries), and per source s = src_of[key] its first record rbeg, and the
// entry range beg, end (nsrc each, zeroed here), in one pass.  scan_words:
// record_scan_words(nrec) words of scratch.  A tile that waits too long for an
// earlier one raises FLAG_SORT in flags.
size_t record_scan_words(int64_t nrec);
int64_t record_scan_tile();  // records per tile of that pass
void grad_record_sources(const uint32_t* skey, const uint32_t* sidx, int64_t nrec,
                         const uint2* crec, const uint32_t* src_of, int64_t nsrc, uint2* srec,
                         uint32_t* recE, unsigned long long* scan_words, uint32_t* rbeg,
                         uint32_t* beg, uint32_t* end, int* flags, cudaStream_t s);
// The same pass with tile 0 withholding its count and every look-back window
// read once: the bounded wait of tile 1 runs out and raises FLAG_SORT (the
// offsets are then wrong; every write stays in bounds).  Only the self-test
// calls it, and nothing reads its output.
void record_scan_wait_selftest(const uint32_t* skey, const uint32_t* sidx, int64_t nrec,
                               const uint2* crec, const uint32_t* src_of, int64_t nsrc,
                               uint2* srec, uint32_t* recE, unsigned long long* scan_words,
                               uint32_t* rbeg, uint32_t* beg, uint32_t* end, int* flags,
                               cudaStream_t s);
// per source s: G_s = sum over its entries of T(r) u_m and Q_s = sum of
// grad phi(r; w_s, u_m) / n_s, r = rho_m - x_s (FP64 results, 3 per source).
// Entry e of source s (beg[s] <= e < end[s]) is particle 32 task + lane of the
// sorted record holding it (recE[r] <= e < recE[r + 1]), its lanes taken in
// rising order.  Each source's entries are cut into items of kGradItemEntries,
// summed one warp each in single precision, the items then added in FP64.
// Scratch: items/item_off (nsrc, nsrc + 1 words), scan_tmp for nsrc, part
// (6 doubles per item; max_items >= nsrc + entries / kGradItemEntries + 1).
constexpr int64_t kGradItemEntries = 1024;
template <typename R>
void grad_source_sums_rec(const vec4<R>* pos, const vec4<R>* u, Tree<R> t, int64_t ncells,
                          int64_t n, const uint2* srec, const uint32_t* recE, int64_t nrec,
                          const uint32_t* rbeg, const uint32_t* beg, const uint32_t* end,
                          uint32_t* items, uint32_t* item_off, uint32_t* scan_tmp, double* part,
                          int64_t max_items, double* G, double* Q, cudaStream_t s);
// per particle p: g_p, q_p = the sums of every cell containing p plus its own
// particle-source sums, then grad_u = -1/2 (h + ds g), grad_pos = -1/2 (f - ds q)
template <typename R>
void grad_finish(Tree<R> t, int64_t ncells, int64_t n, const double* G, const double* Q,
                 const vec4<R>* h, const vec4<R>* f, R ds, vec4<R>* grad_pos, vec4<R>* grad_u,
                 cudaStream_t s);

// Vector-Jacobian product of h and f, source side: per source s,
// G_s = ds sum [T(r) abar_m + grad phi(r; bbar_m, u_m)] (dL/dw_s) and
// Q_s = -ds sum [grad phi(r; abar_m, w_s) + H phi(r; u_m, w_s) bbar_m] / n_s
// (dL/dx_s per member), over the entries of the sorted records; same items,
// order and scratch as grad_source_sums_rec.
template <typename R>
void vjp_source_sums_rec(const vec4<R>* pos, const vec4<R>* u, const vec4<R>* abar,
                         const vec4<R>* bbar, R ds, Tree<R> t, int64_t ncells, int64_t n,
                         const uint2* srec, const uint32_t* recE, int64_t nrec,
                         const uint32_t* rbeg, const uint32_t* beg, const uint32_t* end,
                         uint32_t* items, uint32_t* item_off, uint32_t* scan_tmp, double* part,
                         int64_t max_items, double* G, double* Q, cudaStream_t s);
// dx_p += dxt_p + sum of Q over the cells holding p (and p's own particle
// source), du_p += dut_p + the same for G (accumulated into dx, du).
template <typename R>
void vjp_finish(Tree<R> t, int64_t ncells, int64_t n, const double* G, const double* Q,
                const vec4<R>* dxt, const vec4<R>* dut, vec4<R>* dx, vec4<R>* du, cudaStream_t s);
// out[perm[i]] = in[i] for n records (carries adjoints back through a gather)
template <typename R>
void scatter_records(const uint32_t* perm, int64_t n, const vec4<R>* in, vec4<R>* out,
                     cudaStream_t s);
// sum over n records of component z into *out (FP64, deterministic; tmp holds
// sum_tmp_words(n) doubles)
size_t sum_tmp_words(int64_t n);
template <typename R>
void sum_z(const vec4<R>* v, int64_t n, double* tmp, double* out, cudaStream_t s);

// all pairs exact: the gradient is the negated field and force
template <typename R>
void grad_from_field(const vec4<R>* h, const vec4<R>* f, int64_t n, vec4<R>* grad_pos,
                     vec4<R>* grad_u, cudaStream_t s);

// Barnes-Hut traversal.  h/f (and esr, counts if non-null) in sorted order;
// group = lanes that walk the cell list together (1, 2, 4, 8, 16 or 32);
// work = kWorkSegments task counters (scratch, zeroed by the launcher).
constexpr int kWorkSegments = 1024;
// off = the build's cell offsets (the first cell of position p is off[p]);
// with several systems a particle walks only its own system's cells.
// sched: 0, or one of the launch schedules below (1 .. kNumSchedules), which sets
// the group and, for the plain FP32 walk, the block shape.
struct Schedule {
    int group;          // lanes walking together
    int threads;        // threads per block
    int blocks_per_sm;  // resident blocks the register budget is set for
};
constexpr int kNumSchedules = 10;
constexpr Schedule kSchedules[kNumSchedules] = {
    {1, 128, 12}, {1, 128, 10}, {1, 128, 8}, {1, 256, 6}, {1, 256, 4},
    {1, 64, 24},  {1, 64, 16},  {2, 128, 12}, {4, 128, 12}, {8, 128, 12}};
template <typename R>
void bh_field(const vec4<R>* pos, const vec4<R>* u, int64_t n, Tree<R> t, FieldParams<R> fp,
              vec4<R>* h, vec4<R>* f, R* esr, int4* counts, int* flags, int* work, int group,
              int sched, const uint32_t* off, Segs sg, cudaStream_t s);

// All-pairs sum (Sec. 3.1, Algorithm 1).
template <typename R>
void ap_field(const vec4<R>* pos, const vec4<R>* u, int64_t n, FieldParams<R> fp, vec4<R>* h,
              vec4<R>* f, R* esr, cudaStream_t s);

// Euler-Maruyama step; writes the new state to the second buffers and, if
// partials is non-null, per-block FP64 observables of the old state.
constexpr int kObs = 10;
int integrate_blocks(int64_t n);
template <typename R>
void integrate(int64_t n, const vec4<R>* pos, const vec4<R>* vel, const vec4<R>* u,
               const vec4<R>* om, const uint32_t* id, const vec4<R>* h, const vec4<R>* f,
               const R* esr, DynParams<R> dp, vec4<R>* pos2, vec4<R>* vel2, vec4<R>* u2,
               vec4<R>* om2, uint32_t* id2, double* partials, cudaStream_t s);

// Adjoint of one integrate step (see k_step.cu): adjoints of the outputs in
// xb, vb, ub, wb are replaced by those of the inputs (add_uz first added to
// ub.z); writes the cotangents abar (of h_dip) and bbar (of the interaction
// force) and per-block sums of abar (3 doubles per integrate_blocks(n) block).
template <typename R>
void em_adjoint(int64_t n, const vec4<R>* pos, const vec4<R>* u, const vec4<R>* om,
                const vec4<R>* hdip, DynParams<R> dp, R add_uz, vec4<R>* xb, vec4<R>* vb,
                vec4<R>* ub, vec4<R>* wb, vec4<R>* abar, vec4<R>* bbar, double* partials,
                cudaStream_t s);

// Observables of the state without stepping (per-block partials).
template <typename R>
void observables(int64_t n, const vec4<R>* pos, const vec4<R>* vel, const vec4<R>* u,
                 const vec4<R>* om, const vec4<R>* h, const R* esr, DynParams<R> dp,
                 double* partials, cudaStream_t s);
void reduce_partials(const double* partials, int nblocks, double inv_n, double inertia_half,
                     double* out, cudaStream_t s);
// Advances the device step counter by one (not while FLAG_CAPACITY is raised).
void step_advance(unsigned long long* step, const int* flags, cudaStream_t s);
// sets the device step counter (restoring a saved state)
void step_set(unsigned long long* step, unsigned long long v, cudaStream_t s);

// Layout conversion between caller arrays (n x 3, float or double) and
// records; scatter/gather through the particle ids.
template <typename R, typename I>
void load3(const I* in, int64_t n, vec4<R>* out, cudaStream_t s);
template <typename R>
void fill_zero4(vec4<R>* out, int64_t n, cudaStream_t s);
void iota32(uint32_t* out, int64_t n, cudaStream_t s);
template <typename R, typename O>
void scatter3(const vec4<R>* in, const uint32_t* id, int64_t n, O* out, cudaStream_t s);
template <typename R>
void scatter_counts(const int4* in, const uint32_t* id, int64_t n, int32_t* a, int32_t* p,
                    int32_t* o, cudaStream_t s);

}  // namespace ffk
