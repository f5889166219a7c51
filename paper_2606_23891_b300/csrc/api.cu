// C-ABI entry points of libsph (include/sph.h): argument checks, descriptor
// set-up and kernel launches.  All device code is compiled in this
// translation unit.
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <ctime>
#include <vector>
#include <new>

#include "internal.h"
#include "device.cuh"
#include "pack_kernels.cuh"
#include "physics_kernels.cuh"
#include "store_kernels.cuh"
#include "batch_kernels.cuh"
#include "fp64_kernels.cuh"
#include "list_kernels.cuh"
#include "adjoint_kernels.cuh"
#include "host_batch.cuh"
#include "peak_kernels.cuh"

#include <nvtx3/nvToolsExt.h>

namespace sph {

static thread_local char g_msg[512] = "";

int fail(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return status;
}

static int cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SPH_OK;
    return fail(SPH_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static int launch_check(const char *what) {
    return cuda_check(cudaGetLastError(), what);
}

static int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 148LL * 16) b = 148LL * 16;
    return (int)(b < 1 ? 1 : b);
}

static bool aligned256(const void *p) { return ((uintptr_t)p & 255u) == 0; }

static int check_store(sph_store s) {
    if (!s) return fail(SPH_EINVAL, "NULL store handle");
    if (s->host) return fail(SPH_EINVAL, "store is in host memory: use the *_host calls");
    return SPH_OK;
}

static int check_host_store(sph_store s) {
    if (!s) return fail(SPH_EINVAL, "NULL store handle");
    if (!s->host) return fail(SPH_EINVAL, "store is in device memory: use the device calls");
    return SPH_OK;
}

static int check_tasks(sph_tasks t, int bundle) {
    if (!t) return fail(SPH_EINVAL, "NULL tasks handle");
    if (!t->d_tasks && !t->tdev.empty())
        return fail(SPH_EINVAL, "tasks not uploaded (call sph_tasks_upload)");
    if (bundle < 0 || bundle >= (int64_t)t->bundle_slots.size())
        return fail(SPH_EINVAL, "bundle %d out of range [0, %lld)", bundle,
                    (long long)t->bundle_slots.size());
    return SPH_OK;
}

static int check_loop(int loop) {
    if (loop < SPH_DENSITY || loop > SPH_FORCE) return fail(SPH_EINVAL, "bad loop %d", loop);
    return SPH_OK;
}

static int check_params(const sph_params *p) {
    if (!p) return fail(SPH_EINVAL, "NULL params");
    if (p->reserved != 0) return fail(SPH_EINVAL, "params.reserved must be 0");
    if (!(p->kernel_gamma > 0.0) || !(p->gamma > 1.0))
        return fail(SPH_EINVAL, "params: kernel_gamma > 0 and gamma > 1 required");
    return SPH_OK;
}

// Named host ranges around each stage ("sph/pack/density", ...) for
// timeline profilers; a push and a pop with no tool attached.
struct StageRange {
    explicit StageRange(const char *name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
    StageRange(const StageRange &) = delete;
    StageRange &operator=(const StageRange &) = delete;
};
static const char *stage_name(int stage, int loop) {
    static const char *names[5][3] = {
        {"sph/pack/density", "sph/pack/gradient", "sph/pack/force"},
        {"sph/interact/density", "sph/interact/gradient", "sph/interact/force"},
        {"sph/unpack/density", "sph/unpack/gradient", "sph/unpack/force"},
        {"sph/list_build", "sph/list_build", "sph/list_build"},
        {"sph/adjoint", "sph/adjoint", "sph/adjoint"}};
    return names[stage][loop >= 0 && loop < 3 ? loop : 0];
}
enum { ST_PACK, ST_INTERACT, ST_UNPACK, ST_LIST, ST_ADJOINT };

// Host-side fault injection (tests of the error paths; no device fault):
// the armed site fails on its countdown-th use, once.
static std::atomic<int> g_fault_site{0}, g_fault_countdown{0};

// SPH_FAULT_INJECT=alloc:N or copy:N arms a site when the library loads.
static const int g_fault_env = [] {
    const char *e = getenv("SPH_FAULT_INJECT");
    if (!e) return 0;
    int site = 0;
    if (!strncmp(e, "alloc:", 6)) site = SPH_FAULT_DEVICE_ALLOC;
    else if (!strncmp(e, "copy:", 5)) site = SPH_FAULT_COPY;
    const int n = site ? atoi(strchr(e, ':') + 1) : 0;
    if (site && n > 0) {
        g_fault_countdown.store(n);
        g_fault_site.store(site);
    } else {
        fprintf(stderr, "libsph: SPH_FAULT_INJECT=%s not understood (alloc:N or copy:N)\n", e);
    }
    return site;
}();

static bool fault_fires(int site) {
    if (g_fault_site.load() != site) return false;
    if (g_fault_countdown.fetch_sub(1) != 1) return false;
    g_fault_site.store(0);
    return true;
}

// Device allocation and upload of plan metadata, failing where injected.
static int upload_meta(void **dst, const void *src, size_t bytes, const char *what) {
    if (bytes == 0) return SPH_OK;
    if (fault_fires(SPH_FAULT_DEVICE_ALLOC) || cudaMalloc(dst, bytes) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return fail(SPH_ENOMEM, "device allocation of %s (%zu bytes)", what, bytes);
    }
    if (fault_fires(SPH_FAULT_COPY))
        return fail(SPH_ECUDA, "%s: injected copy failure", what);
    if (!src) return cuda_check(cudaMemset(*dst, 0, bytes), what);
    return cuda_check(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), what);
}

// Store address of (field, comp); every field exists in every layout.
static CompPtr at(sph_store s, int field, int comp) {
    CompPtr c{nullptr, 0};
    locate(s->layout, s->mem, field, comp, &c);
    return c;
}

// The copy of (field, comp) that the pack of `loop` reads.
static CompPtr at_view(sph_store s, int field, int comp, int loop) {
    CompPtr c{nullptr, 0};
    locate_view(s->layout, s->mem, field, comp, loop, &c);
    return c;
}

static void lanes(int loop, int in_or_out, int64_t S, char *buf, char **out, int *nl) {
    int64_t off[16];
    int64_t sz[16];
    *nl = lane_sizes(loop, in_or_out, sz);
    lane_offsets(loop, in_or_out, S, off);
    for (int k = 0; k < *nl; ++k) out[k] = buf + off[k];
}

static int check_bundle_store(sph_store s, sph_tasks t) {
    if (s->n != t->n)
        return fail(SPH_EINVAL, "store has %lld particles, tasks %lld", (long long)s->n,
                    (long long)t->n);
    return SPH_OK;
}

template <int LOOP, int T>
int launch_binteract(const BInteractArgs &a, cudaStream_t st) {
    static int cached_dev = -1, grid_max = 0;
    int dev = 0;
    if (int rc = cuda_check(cudaGetDevice(&dev), "get device")) return rc;
    if (cached_dev != dev) {
        int per_sm = 0, sms = 0;
        if (int rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                    &per_sm, k_binteract<LOOP, T>, T, 0),
                                "occupancy"))
            return rc;
        if (int rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                                "SM count"))
            return rc;
        grid_max = (per_sm > 0 ? per_sm : 1) * sms;
        cached_dev = dev;
    }
    const int g = a.nitems < grid_max ? a.nitems : grid_max;
    if (g <= 0) return SPH_OK;
    k_binteract<LOOP, T><<<g, T, 0, st>>>(a);
    return launch_check("batch interaction kernel");
}

// Persistent launch: as many CTAs as fit on the device at once (occupancy
// looked up once per kernel and device), at most one per work item.
template <typename Kernel, typename... Args>
int launch_persistent(Kernel kernel, int threads, int nitems, cudaStream_t st, const char *what,
                      Args... args) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> grid_of;
    int dev = 0;
    if (int rc = cuda_check(cudaGetDevice(&dev), "get device")) return rc;
    int grid_max = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto key = std::make_pair((const void *)kernel, dev);
        auto itg = grid_of.find(key);
        if (itg == grid_of.end()) {
            int per_sm = 0, sms = 0;
            if (int rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel,
                                                                                  threads, 0),
                                    "occupancy"))
                return rc;
            if (int rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount,
                                                           dev),
                                    "SM count"))
                return rc;
            itg = grid_of.emplace(key, (per_sm > 0 ? per_sm : 1) * sms).first;
        }
        grid_max = itg->second;
    }
    const int g = nitems < grid_max ? nitems : grid_max;
    if (g <= 0) return SPH_OK;
    kernel<<<g, threads, 0, st>>>(args...);
    return launch_check(what);
}

template <int LOOP, int W>
int dispatch_bloop_w(int threads, const BInteractArgs &a, const ListView &L, long long item0,
                     cudaStream_t st) {
    if (threads == 64)
        return launch_persistent(k_bloop<LOOP, 64, W>, 64, a.nitems, st, "list loop", a, L,
                                 item0);
    if (threads == 256)
        return launch_persistent(k_bloop<LOOP, 256, W>, 256, a.nitems, st, "list loop", a, L,
                                 item0);
    return launch_persistent(k_bloop<LOOP, 128, W>, 128, a.nitems, st, "list loop", a, L, item0);
}

// The list loops' register caps by plan kind (kLLoopWarpsGrid / kLLoopWarpsTree).
// The force loop on grid plans runs one CTA per SM over chunks of
// consecutive items (k_bloop's CH mode): 6.35 against 6.57 ms at Gresho256.
// The same mode made the density and gradient loops slower (4.69 / 4.58
// against 3.99 / 3.79 ms), so they keep the launch-wide item queue.
template <int LOOP>
int dispatch_bloop(sph_batch b, const BInteractArgs &a, const ListView &L, long long item0,
                   cudaStream_t st) {
    if constexpr (LOOP != SPH_FORCE)
        if (b->kind == 1)
            return dispatch_bloop_w<LOOP, kLLoopWarpsTree>(b->threads, a, L, item0, st);
    if constexpr (LOOP == SPH_FORCE)
        if (b->kind == 0)
            return launch_persistent(
                k_bloop<LOOP, 32 * kLLoopWarpsForce, kLLoopWarpsForce, false, true>,
                32 * kLLoopWarpsForce, a.nitems, st, "list loop", a, L, item0);
    return dispatch_bloop_w<LOOP, kLLoopWarpsGrid<LOOP>>(b->threads, a, L, item0, st);
}

// The FP64-separation list loops of the precision study (more registers:
// capped for 28 warps).
template <int LOOP>
int dispatch_bloop64(sph_batch b, const BInteractArgs &a, const ListView &L, long long item0,
                     cudaStream_t st) {
    constexpr int W = kLLoopWarpsForce;
    if (b->threads == 64)
        return launch_persistent(k_bloop<LOOP, 64, W, true>, 64, a.nitems, st, "list loop (FP64 "
                                 "separations)", a, L, item0);
    if (b->threads == 256)
        return launch_persistent(k_bloop<LOOP, 256, W, true>, 256, a.nitems, st, "list loop "
                                 "(FP64 separations)", a, L, item0);
    return launch_persistent(k_bloop<LOOP, 128, W, true>, 128, a.nitems, st, "list loop (FP64 "
                             "separations)", a, L, item0);
}

template <bool FIXED>
inline int dispatch_blist_p(int threads, const BInteractArgs &a, const ListView &L,
                            long long item0, cudaStream_t st) {
    unsigned long long *none = nullptr;
    if (threads == 64)
        return launch_persistent(k_blist<64, FIXED>, 64, a.nitems, st, "list build", a, L, item0,
                                 none);
    if (threads == 256)
        return launch_persistent(k_blist<256, FIXED>, 256, a.nitems, st, "list build", a, L,
                                 item0, none);
    return launch_persistent(k_blist<128, FIXED>, 128, a.nitems, st, "list build", a, L, item0,
                             none);
}

// The list build takes the fixed-point path where the plan allows it, and
// the symmetric build (two passes) where the plan holds its data.
template <bool COUNT>
int dispatch_blist_sym(int threads, const BInteractArgs &a, const ListView &L, long long item0,
                       unsigned long long *cnt, cudaStream_t st) {
    const char *w1 = "list build (symmetric, first pass)", *w2 = "list build (second pass)";
    int rc;
    if (threads == 64)
        rc = launch_persistent(k_blist<64, true, COUNT, true>, 64, a.nitems, st, w1, a, L, item0,
                               cnt);
    else if (threads == 256)
        rc = launch_persistent(k_blist<256, true, COUNT, true>, 256, a.nitems, st, w1, a, L,
                               item0, cnt);
    else
        rc = launch_persistent(k_blist<128, true, COUNT, true>, 128, a.nitems, st, w1, a, L,
                               item0, cnt);
    if (rc) return rc;
    if ((rc = cuda_check(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st),
                         "reset work queue")))
        return rc;
    if (threads == 64)
        return launch_persistent(k_blist_rev<64, COUNT>, 64, a.nitems, st, w2, a, L, item0, cnt);
    if (threads == 256)
        return launch_persistent(k_blist_rev<256, COUNT>, 256, a.nitems, st, w2, a, L, item0,
                                 cnt);
    return launch_persistent(k_blist_rev<128, COUNT>, 128, a.nitems, st, w2, a, L, item0, cnt);
}

inline int dispatch_blist(sph_batch b, const BInteractArgs &a, const ListView &L,
                          long long item0, cudaStream_t st) {
    if (b->sym && b->sym_on)
        return dispatch_blist_sym<false>(b->threads, a, L, item0, nullptr, st);
    if (b->fixed_build) return dispatch_blist_p<true>(b->threads, a, L, item0, st);
    return dispatch_blist_p<false>(b->threads, a, L, item0, st);
}

// The counting variant of the list build (measurement only), at the plan's
// block size of 128 threads or 64 / 256 as configured.
template <bool FIXED>
inline int dispatch_blist_count_p(int threads, const BInteractArgs &a, const ListView &L,
                                  long long item0, unsigned long long *cnt, cudaStream_t st) {
    if (threads == 64)
        return launch_persistent(k_blist<64, FIXED, true>, 64, a.nitems, st, "list count", a, L,
                                 item0, cnt);
    if (threads == 256)
        return launch_persistent(k_blist<256, FIXED, true>, 256, a.nitems, st, "list count", a,
                                 L, item0, cnt);
    return launch_persistent(k_blist<128, FIXED, true>, 128, a.nitems, st, "list count", a, L,
                             item0, cnt);
}

template <int LOOP>
int dispatch_binteract(int threads, const BInteractArgs &a, cudaStream_t st) {
    if (threads == 64) return launch_binteract<LOOP, 64>(a, st);
    if (threads == 256) return launch_binteract<LOOP, 256>(a, st);
    return launch_binteract<LOOP, 128>(a, st);
}

}  // namespace sph

using namespace sph;

extern "C" {

const char *sph_version(void) { return "sph-b300 0.1 (sm_103a)"; }

const char *sph_last_error(void) { return g_msg; }

size_t sph_store_bytes(int64_t n, int layout, uint64_t seed) {
    if (n < 0) return 0;
    Layout L;
    if (build_layout(layout, seed, n, &L) != SPH_OK) return 0;
    return (size_t)layout_bytes(L, n);
}

int sph_layout_group_count(int layout, uint64_t seed) {
    Layout L;
    if (build_layout(layout, seed, 0, &L) != SPH_OK) return -1;
    return (int)L.groups.size();
}

int sph_layout_describe(int layout, uint64_t seed, int group, int32_t *nmem,
                        int32_t *field_ids, int32_t *comps, int32_t *offsets,
                        int32_t *record_bytes) {
    Layout L;
    if (build_layout(layout, seed, 0, &L) != SPH_OK)
        return fail(SPH_EINVAL, "bad layout %d", layout);
    if (group < 0 || group >= (int)L.groups.size())
        return fail(SPH_EINVAL, "group %d out of range", group);
    const Group &g = L.groups[group];
    if (nmem) *nmem = (int32_t)g.mem.size();
    for (size_t k = 0; k < g.mem.size(); ++k) {
        if (field_ids) field_ids[k] = g.mem[k].field;
        if (comps) comps[k] = g.mem[k].comp;
        if (offsets) offsets[k] = g.mem[k].offset;
    }
    if (record_bytes) *record_bytes = g.record;
    return SPH_OK;
}

int sph_store_create(int64_t n, int layout, uint64_t seed, void *dev_mem, size_t bytes,
                     sph_store *out) {
    if (!out) return fail(SPH_EINVAL, "NULL out");
    *out = nullptr;
    if (n < 0 || n > INT32_MAX) return fail(SPH_EINVAL, "bad particle count %lld", (long long)n);
    Layout L;
    if (build_layout(layout, seed, n, &L) != SPH_OK)
        return fail(SPH_EINVAL, "bad layout %d", layout);
    const int64_t need = layout_bytes(L, n);
    if ((int64_t)bytes < need)
        return fail(SPH_EINVAL, "store needs %lld bytes, got %zu", (long long)need, bytes);
    if (need > 0 && (!dev_mem || !aligned256(dev_mem)))
        return fail(SPH_EINVAL, "store memory must be a 256-byte aligned device pointer");
    sph_store s = new (std::nothrow) sph_store_s;
    if (!s) return fail(SPH_ENOMEM, "store handle");
    s->n = n;
    s->layout = L;
    s->mem = (char *)dev_mem;
    s->bytes = bytes;
    if (need > 0) {
        int rc = cuda_check(cudaMemset(dev_mem, 0, (size_t)need), "store zero-fill");
        if (rc) {
            delete s;
            return rc;
        }
    }
    *out = s;
    return SPH_OK;
}

int sph_store_destroy(sph_store s) {
    delete s;
    return SPH_OK;
}

static int copy_fields(sph_store s, const sph_fields *f, const int64_t *perm, void *stream,
                       int to_store) {
    if (int rc = check_store(s)) return rc;
    if (!f) return fail(SPH_EINVAL, "NULL fields");
    if (s->n == 0) return SPH_OK;
    void *const *ptrs = reinterpret_cast<void *const *>(f);
    const int nfields = (int)(sizeof(sph_fields) / sizeof(void *));
    cudaStream_t st = (cudaStream_t)stream;
    // every requested component in one launch (a second one past kCopyMax)
    CopyArgs a{};
    auto flush = [&]() -> int {
        if (a.ncomp == 0) return SPH_OK;
        k_copy_fields<<<grid_for(s->n, 256), 256, 0, st>>>(a, perm, s->n, to_store);
        a.ncomp = 0;
        return launch_check("copy fields");
    };
    for (int fid = 0; fid < nfields && fid < F_BALLAST; ++fid) {
        const char *p = (const char *)ptrs[fid];
        if (!p) continue;
        const int elem = kFields[fid].elem, cnt = kFields[fid].count;
        for (int c = 0; c < cnt; ++c) {
            // into the store: every copy of a replicated field; out: the first
            CompPtr dst[4];
            const int ncopy = to_store ? locate_all(s->layout, s->mem, fid, c, dst, 4)
                                       : (int)locate(s->layout, s->mem, fid, c, dst);
            for (int k = 0; k < ncopy; ++k) {
                if (a.ncomp == kCopyMax)
                    if (int rc = flush()) return rc;
                a.c[a.ncomp++] = CopyComp{p, elem * cnt, c * elem, elem, dst[k]};
            }
        }
    }
    return flush();
}

int sph_store_convert(sph_store dst, sph_store src, void *stream) {
    if (int rc = check_store(dst)) return rc;
    if (int rc = check_store(src)) return rc;
    if (dst->n != src->n) return fail(SPH_EINVAL, "stores differ in particle count");
    if (dst == src) return SPH_OK;
    ConvArgs a{};
    for (int fid = 0; fid < F_NUM; ++fid) {
        const int elem = kFields[fid].elem, cnt = kFields[fid].count;
        for (int c = 0; c < cnt; ++c) {
            CompPtr from{nullptr, 0}, to[4];
            if (!locate(src->layout, src->mem, fid, c, &from)) continue;
            const int nto = locate_all(dst->layout, dst->mem, fid, c, to, 4);
            for (int k = 0; k < nto; ++k) {
                if (a.ncomp == (int)(sizeof(a.c) / sizeof(a.c[0])))
                    return fail(SPH_EUNSUPPORTED, "layout has too many components to convert");
                a.c[a.ncomp++] = ConvComp{to[k], from, elem};
            }
        }
    }
    if (src->n == 0) return SPH_OK;
    k_convert<<<grid_for(src->n, 256), 256, 0, (cudaStream_t)stream>>>(a, src->n);
    return launch_check("store convert");
}

int sph_store_import(sph_store s, const sph_fields *dev_src, const int64_t *dev_perm,
                     void *stream) {
    return copy_fields(s, dev_src, dev_perm, stream, 1);
}

int sph_store_export(sph_store s, const sph_fields *dev_dst, const int64_t *dev_perm,
                     void *stream) {
    return copy_fields(s, dev_dst, dev_perm, stream, 0);
}

}  // extern "C"

// ---- end-to-end host I/O ----------------------------------------------------
struct sph_hostio_s {
    sph_store s = nullptr;
    const int64_t *perm = nullptr;
    int nin = 0, nout = 0;
    int fin[F_BALLAST], fout[F_BALLAST];   // selected field ids
    size_t fbytes[F_BALLAST];              // bytes of each field for n particles
    char *stage_in[2][F_BALLAST], *stage_out[2][F_BALLAST];
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    cudaEvent_t in_ready[2], in_free[2], out_ready[2], out_free[2];
    int nev = 0;
    long long k = 0;     // steps begun
    bool open = false;   // a step was begun and not yet ended
};

namespace sph {

static int hostio_select(const sph_fields *sel, int *ids) {
    if (!sel) return 0;
    void *const *p = reinterpret_cast<void *const *>(sel);
    int n = 0;
    for (int f = 0; f < F_BALLAST; ++f)
        if (p[f]) ids[n++] = f;
    return n;
}

static size_t hostio_field_bytes(int64_t n, int f) {
    return (size_t)n * kFields[f].elem * kFields[f].count;
}

static size_t r256(size_t b) { return (b + 255) / 256 * 256; }

static size_t hostio_set_bytes(int64_t n, const int *ids, int nf) {
    size_t b = 0;
    for (int k = 0; k < nf; ++k) b += r256(hostio_field_bytes(n, ids[k]));
    return b;
}

// The host arrays of a step must be exactly the selected fields, each in
// page-locked memory (a pageable source would turn the copies synchronous).
static int hostio_host_ptrs(const sph_fields *f, const int *ids, int nf, void **out,
                            const char *what) {
    if (!f) return fail(SPH_EINVAL, "%s: NULL fields", what);
    void *const *p = reinterpret_cast<void *const *>(f);
    int want[F_BALLAST] = {0};
    for (int k = 0; k < nf; ++k) want[ids[k]] = 1;
    for (int fid = 0; fid < F_BALLAST; ++fid) {
        if ((p[fid] != nullptr) != (want[fid] != 0))
            return fail(SPH_EINVAL, "%s: field %d %s", what, fid,
                        want[fid] ? "is selected but NULL" : "was not selected at create");
    }
    for (int k = 0; k < nf; ++k) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p[ids[k]]) != cudaSuccess) {
            cudaGetLastError();
            return fail(SPH_EINVAL, "%s: field %d is not a host pointer CUDA knows", what, ids[k]);
        }
        if (at.type != cudaMemoryTypeHost)
            return fail(SPH_EINVAL, "%s: field %d must be page-locked host memory", what, ids[k]);
        out[k] = p[ids[k]];
    }
    return SPH_OK;
}

static void hostio_fields(char *const *stage, const int *ids, int nf, sph_fields *out) {
    std::memset(out, 0, sizeof(*out));
    void **p = reinterpret_cast<void **>(out);
    for (int k = 0; k < nf; ++k) p[ids[k]] = stage[k];
}

}  // namespace sph

extern "C" {

size_t sph_hostio_bytes(int64_t n, const sph_fields *in_sel, const sph_fields *out_sel) {
    if (n < 0) return 0;
    int fi[F_BALLAST], fo[F_BALLAST];
    const int ni = hostio_select(in_sel, fi), no = hostio_select(out_sel, fo);
    return 2 * (hostio_set_bytes(n, fi, ni) + hostio_set_bytes(n, fo, no));
}

int sph_hostio_create(sph_store s, const int64_t *dev_perm, const sph_fields *in_sel,
                      const sph_fields *out_sel, void *dev_staging, size_t bytes,
                      void *copy_in_stream, void *copy_out_stream, sph_hostio *out) {
    if (!out) return fail(SPH_EINVAL, "NULL out");
    *out = nullptr;
    if (int rc = check_store(s)) return rc;
    if (!dev_perm && s->n > 0) return fail(SPH_EINVAL, "NULL permutation");
    if (!aligned256(dev_staging)) return fail(SPH_EINVAL, "staging must be 256-byte aligned");
    auto *io = new (std::nothrow) sph_hostio_s();
    if (!io) return fail(SPH_ENOMEM, "host I/O handle");
    io->s = s;
    io->perm = dev_perm;
    io->nin = hostio_select(in_sel, io->fin);
    io->nout = hostio_select(out_sel, io->fout);
    if (io->nin + io->nout == 0) {
        delete io;
        return fail(SPH_EINVAL, "no field selected");
    }
    const size_t need = sph_hostio_bytes(s->n, in_sel, out_sel);
    if (bytes < need || (need > 0 && !dev_staging)) {
        delete io;
        return fail(SPH_EINVAL, "staging holds %zu bytes, needs %zu", bytes, need);
    }
    char *p = (char *)dev_staging;
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < io->nin; ++k) {
            io->stage_in[b][k] = p;
            p += r256(hostio_field_bytes(s->n, io->fin[k]));
        }
        for (int k = 0; k < io->nout; ++k) {
            io->stage_out[b][k] = p;
            p += r256(hostio_field_bytes(s->n, io->fout[k]));
        }
    }
    for (int f = 0; f < F_BALLAST; ++f) io->fbytes[f] = hostio_field_bytes(s->n, f);
    io->copy_in = (cudaStream_t)copy_in_stream;
    io->copy_out = (cudaStream_t)copy_out_stream;
    cudaEvent_t *ev[8] = {&io->in_ready[0], &io->in_ready[1], &io->in_free[0], &io->in_free[1],
                          &io->out_ready[0], &io->out_ready[1], &io->out_free[0],
                          &io->out_free[1]};
    for (int e = 0; e < 8; ++e) {
        if (int rc = cuda_check(cudaEventCreateWithFlags(ev[e], cudaEventDisableTiming),
                                "host I/O event")) {
            for (int q = 0; q < io->nev; ++q) cudaEventDestroy(*ev[q]);
            delete io;
            return rc;
        }
        io->nev = e + 1;
    }
    *out = io;
    return SPH_OK;
}

int sph_hostio_begin(sph_hostio io, const sph_fields *host_in, void *stream) {
    if (!io) return fail(SPH_EINVAL, "NULL host I/O handle");
    if (io->open) return fail(SPH_EINVAL, "host I/O: the previous step was not ended");
    void *src[F_BALLAST];
    if (int rc = hostio_host_ptrs(host_in, io->fin, io->nin, src, "host I/O begin")) return rc;
    const int b = (int)(io->k & 1);
    cudaStream_t st = (cudaStream_t)stream;
    // staging set b was last read by the import of step k - 2
    if (int rc = cuda_check(cudaStreamWaitEvent(io->copy_in, io->in_free[b], 0), "wait"))
        return rc;
    for (int k = 0; k < io->nin; ++k)
        if (int rc = cuda_check(cudaMemcpyAsync(io->stage_in[b][k], src[k],
                                                io->fbytes[io->fin[k]], cudaMemcpyHostToDevice,
                                                io->copy_in),
                                "host I/O H2D"))
            return rc;
    if (int rc = cuda_check(cudaEventRecord(io->in_ready[b], io->copy_in), "record")) return rc;
    if (int rc = cuda_check(cudaStreamWaitEvent(st, io->in_ready[b], 0), "wait")) return rc;
    if (io->nin > 0) {
        sph_fields F;
        hostio_fields(io->stage_in[b], io->fin, io->nin, &F);
        if (int rc = sph_store_import(io->s, &F, io->perm, stream)) return rc;
    }
    if (int rc = cuda_check(cudaEventRecord(io->in_free[b], st), "record")) return rc;
    io->open = true;
    return SPH_OK;
}

int sph_hostio_end(sph_hostio io, const sph_fields *host_out, void *stream) {
    if (!io) return fail(SPH_EINVAL, "NULL host I/O handle");
    if (!io->open) return fail(SPH_EINVAL, "host I/O: no step was begun");
    void *dst[F_BALLAST];
    if (int rc = hostio_host_ptrs(host_out, io->fout, io->nout, dst, "host I/O end")) return rc;
    const int b = (int)(io->k & 1);
    cudaStream_t st = (cudaStream_t)stream;
    // staging set b was last read by the D2H copies of step k - 2
    if (int rc = cuda_check(cudaStreamWaitEvent(st, io->out_free[b], 0), "wait")) return rc;
    if (io->nout > 0) {
        sph_fields F;
        hostio_fields(io->stage_out[b], io->fout, io->nout, &F);
        if (int rc = sph_store_export(io->s, &F, io->perm, stream)) return rc;
    }
    if (int rc = cuda_check(cudaEventRecord(io->out_ready[b], st), "record")) return rc;
    if (int rc = cuda_check(cudaStreamWaitEvent(io->copy_out, io->out_ready[b], 0), "wait"))
        return rc;
    for (int k = 0; k < io->nout; ++k)
        if (int rc = cuda_check(cudaMemcpyAsync(dst[k], io->stage_out[b][k],
                                                io->fbytes[io->fout[k]], cudaMemcpyDeviceToHost,
                                                io->copy_out),
                                "host I/O D2H"))
            return rc;
    if (int rc = cuda_check(cudaEventRecord(io->out_free[b], io->copy_out), "record")) return rc;
    io->open = false;
    ++io->k;
    return SPH_OK;
}

int sph_hostio_drain(sph_hostio io, void *stream) {
    if (!io) return fail(SPH_EINVAL, "NULL host I/O handle");
    if (io->k == 0) return SPH_OK;
    const int b = (int)((io->k - 1) & 1);
    return cuda_check(cudaStreamWaitEvent((cudaStream_t)stream, io->out_free[b], 0), "wait");
}

int sph_hostio_info(sph_hostio io, int64_t info[3]) {
    if (!io || !info) return fail(SPH_EINVAL, "NULL argument");
    int64_t hin = 0, hout = 0;
    for (int k = 0; k < io->nin; ++k) hin += (int64_t)io->fbytes[io->fin[k]];
    for (int k = 0; k < io->nout; ++k) hout += (int64_t)io->fbytes[io->fout[k]];
    info[0] = hin;
    info[1] = hout;
    info[2] = io->k;
    return SPH_OK;
}

int sph_hostio_destroy(sph_hostio io) {
    if (!io) return SPH_OK;
    cudaEvent_t ev[8] = {io->in_ready[0], io->in_ready[1], io->in_free[0], io->in_free[1],
                         io->out_ready[0], io->out_ready[1], io->out_free[0], io->out_free[1]};
    for (int e = 0; e < io->nev; ++e) cudaEventDestroy(ev[e]);
    delete io;
    return SPH_OK;
}

// ---- arithmetic-peak microbenchmarks ----------------------------------------
int sph_peak_run(int kind, int64_t iters, void *dev_sink, void *stream, double *flops_out) {
    if (kind < 0 || kind > 2) return fail(SPH_EINVAL, "bad peak kind %d", kind);
    if (iters <= 0 || !dev_sink || !aligned256(dev_sink))
        return fail(SPH_EINVAL, "iters must be > 0 and the sink a 256-byte aligned pointer");
    int dev = 0, sms = 0;
    if (int rc = cuda_check(cudaGetDevice(&dev), "device")) return rc;
    if (int rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                            "SM count"))
        return rc;
    const int blocks = 8 * sms, threads = 256;   // 64 warps per SM
    cudaStream_t st = (cudaStream_t)stream;
    if (kind == 0)
        k_peak<float, 0><<<blocks, threads, 0, st>>>(iters, 1.0f, (float *)dev_sink);
    else if (kind == 1)
        k_peak<double, 1><<<blocks, threads, 0, st>>>(iters, 1.0, (double *)dev_sink);
    else
        k_peak<double, 2><<<blocks, threads, 0, st>>>(iters, 1.0, (double *)dev_sink);
    if (flops_out)
        *flops_out = (double)blocks * threads * (double)iters * kPeakUnroll * kPeakChains *
                     (kind == 2 ? 1.0 : 2.0);
    return launch_check("peak microbenchmark");
}

int sph_tasks_build(int64_t n, const double *host_x, const float *host_h,
                    const sph_grid_params *gp, int64_t *host_perm_out, sph_tasks *out) {
    if (!out) return fail(SPH_EINVAL, "NULL out");
    *out = nullptr;
    sph_tasks t = new (std::nothrow) sph_tasks_s;
    if (!t) return fail(SPH_ENOMEM, "tasks handle");
    int rc;
    try {
        rc = build_tasks(n, host_x, host_h, gp, host_perm_out, t);
    } catch (const std::bad_alloc &) {
        rc = fail(SPH_ENOMEM, "tasks_build: host allocation failed");
    }
    if (rc) {
        delete t;
        return rc;
    }
    *out = t;
    return SPH_OK;
}

static void free_device(sph_tasks t) {
    if (t->d_tasks) cudaFree(t->d_tasks);
    if (t->d_ucells) cudaFree(t->d_ucells);
    if (t->d_entries) cudaFree(t->d_entries);
    t->d_tasks = nullptr;
    t->d_ucells = nullptr;
    t->d_entries = nullptr;
}

int sph_tasks_upload(sph_tasks t) {
    if (!t) return fail(SPH_EINVAL, "NULL tasks handle");
    free_device(t);
    int rc;
    auto up = [&](void **dst, const void *src, size_t bytes, const char *what) -> int {
        return upload_meta(dst, src, bytes, what);
    };
    if ((rc = up((void **)&t->d_tasks, t->tdev.data(), t->tdev.size() * sizeof(TaskDev),
                 "tasks")) ||
        (rc = up((void **)&t->d_ucells, t->ucells.data(), t->ucells.size() * sizeof(UCellDev),
                 "unpack cells")) ||
        (rc = up((void **)&t->d_entries, t->entries.data(), t->entries.size() * sizeof(int32_t),
                 "unpack entries"))) {
        free_device(t);
        return rc;
    }
    cudaGetDevice(&t->device);
    return SPH_OK;
}

int sph_tasks_info(sph_tasks t, int64_t info[10]) {
    if (!t || !info) return fail(SPH_EINVAL, "NULL argument");
    int64_t total = 0, big = 0, nonempty = 0;
    for (int64_t s : t->bundle_slots) {
        total += s;
        if (s > big) big = s;
    }
    for (size_t c = 0; c + 1 < t->cell_start.size(); ++c)
        if (t->cell_start[c + 1] > t->cell_start[c]) nonempty++;
    info[0] = t->ncell[0];
    info[1] = t->ncell[1];
    info[2] = t->ncell[2];
    info[3] = (int64_t)t->ci.size();
    info[4] = (int64_t)t->bundle_slots.size();
    info[5] = total;
    info[6] = big;
    info[7] = nonempty;
    info[8] = t->n;
    info[9] = t->max_cell;
    return SPH_OK;
}

int sph_tasks_get(sph_tasks t, int32_t *ci, int32_t *cj, int8_t *shift, int64_t *cell_start,
                  int64_t *bundle_start) {
    if (!t) return fail(SPH_EINVAL, "NULL tasks handle");
    if (ci) memcpy(ci, t->ci.data(), t->ci.size() * sizeof(int32_t));
    if (cj) memcpy(cj, t->cj.data(), t->cj.size() * sizeof(int32_t));
    if (shift) memcpy(shift, t->shift.data(), t->shift.size());
    if (cell_start) memcpy(cell_start, t->cell_start.data(), t->cell_start.size() * sizeof(int64_t));
    if (bundle_start)
        memcpy(bundle_start, t->bundle_start.data(), t->bundle_start.size() * sizeof(int64_t));
    return SPH_OK;
}

size_t sph_buffer_bytes(sph_tasks t, int loop, int in_or_out) {
    if (!t || loop < SPH_DENSITY || loop > SPH_FORCE || (in_or_out != 0 && in_or_out != 1))
        return 0;
    int64_t big = 0;
    for (int64_t s : t->bundle_slots) big = s > big ? s : big;
    int64_t off[16];
    return (size_t)lane_offsets(loop, in_or_out, big, off);
}

int sph_tasks_destroy(sph_tasks t) {
    if (!t) return SPH_OK;
    free_device(t);
    delete t;
    return SPH_OK;
}

int sph_init(sph_store s, int loop, const sph_params *p, void *stream) {
    if (int rc = check_store(s)) return rc;
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (s->n == 0) return SPH_OK;
    InitArgs a{};
    int k = 0;
    if (loop == SPH_DENSITY) {
        a.out[k++] = at(s, F_RHO, 0);
        a.out[k++] = at(s, F_RHODH, 0);
        a.out[k++] = at(s, F_WCOUNT, 0);
        a.out[k++] = at(s, F_WCOUNTDH, 0);
        a.out[k++] = at(s, F_DIVV, 0);
        for (int c = 0; c < 3; ++c) a.out[k++] = at(s, F_ROTV, c);
    } else if (loop == SPH_GRADIENT) {
        a.out[k++] = at(s, F_VSIGG, 0);
        a.out[k++] = at(s, F_LAPU, 0);
    } else {
        for (int c = 0; c < 3; ++c) a.out[k++] = at(s, F_A, c);
        a.out[k++] = at(s, F_UDT, 0);
        a.out[k++] = at(s, F_HDT, 0);
        a.out[k++] = at(s, F_VSIG, 0);
        a.use_tb = 1;
        a.tb = at(s, F_TBIN, 0);
        a.active_bin = p->active_bin;
    }
    a.nout = k;
    k_init<<<grid_for(s->n, 256), 256, 0, (cudaStream_t)stream>>>(a, s->n);
    return launch_check("init");
}

int sph_pack(sph_store s, sph_tasks t, int loop, int bundle, void *dev_buf_in, void *stream) {
    StageRange range_(stage_name(ST_PACK, loop));
    if (int rc = check_store(s)) return rc;
    if (int rc = check_tasks(t, bundle)) return rc;
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_bundle_store(s, t)) return rc;
    if (!dev_buf_in || !aligned256(dev_buf_in))
        return fail(SPH_EINVAL, "pack buffer must be a 256-byte aligned device pointer");
    const int64_t t0 = t->bundle_start[bundle], nt = t->bundle_start[bundle + 1] - t0;
    PackArgs a{};
    a.tasks = t->d_tasks + t0;
    int nl;
    lanes(loop, 0, t->bundle_slots[bundle], (char *)dev_buf_in, a.lane, &nl);
    const int roles[R_NUM][2] = {{F_X, 0}, {F_X, 1}, {F_X, 2}, {F_V, 0}, {F_V, 1},
                                 {F_V, 2}, {F_MASS, 0}, {F_H, 0}, {F_U, 0}, {F_RHO, 0},
                                 {F_FGRADH, 0}, {F_BALS, 0}, {F_AVISC, 0}, {F_ADIFF, 0},
                                 {F_TBIN, 0}};
    for (int r = 0; r < R_NUM; ++r) a.src[r] = at_view(s, roles[r][0], roles[r][1], loop);
    for (int d = 0; d < 3; ++d) a.box[d] = t->box[d];
    cudaStream_t st = (cudaStream_t)stream;
    if (nt == 0) return SPH_OK;
    if (loop == SPH_DENSITY) k_pack<SPH_DENSITY><<<(unsigned)nt, 128, 0, st>>>(a);
    else if (loop == SPH_GRADIENT) k_pack<SPH_GRADIENT><<<(unsigned)nt, 128, 0, st>>>(a);
    else k_pack<SPH_FORCE><<<(unsigned)nt, 128, 0, st>>>(a);
    return launch_check("pack");
}

static int interact(sph_tasks t, int loop, int bundle, const void *in, void *out,
                    const sph_params *p, unsigned long long *count, void *stream) {
    StageRange range_(stage_name(ST_INTERACT, loop));
    if (int rc = check_tasks(t, bundle)) return rc;
    if (int rc = check_params(p)) return rc;
    if (!in || !aligned256(in))
        return fail(SPH_EINVAL, "pack buffer must be a 256-byte aligned device pointer");
    if (!count && (!out || !aligned256(out)))
        return fail(SPH_EINVAL, "result buffer must be a 256-byte aligned device pointer");
    const int64_t t0 = t->bundle_start[bundle], nt = t->bundle_start[bundle + 1] - t0;
    PhysArgs a{};
    a.tasks = t->d_tasks + t0;
    int nl;
    char *inl[16];
    lanes(loop, 0, t->bundle_slots[bundle], (char *)in, inl, &nl);
    for (int k = 0; k < nl; ++k) a.in[k] = inl[k];
    if (!count) lanes(loop, 1, t->bundle_slots[bundle], (char *)out, a.out, &nl);
    a.kernel_gamma = (float)p->kernel_gamma;
    a.gamma = (float)p->gamma;
    a.beta = (float)p->beta_visc;
    double bmax = t->box[0] > t->box[1] ? t->box[0] : t->box[1];
    bmax = bmax > t->box[2] ? bmax : t->box[2];
    a.delta = (float)(4e-6 * bmax);
    a.active_bin = p->active_bin;
    a.count = count;
    cudaStream_t st = (cudaStream_t)stream;
    if (nt == 0) return SPH_OK;
    const unsigned g = (unsigned)nt;
    if (count) {
        if (loop == SPH_DENSITY) k_interact<SPH_DENSITY, true><<<g, kThreads, 0, st>>>(a);
        else if (loop == SPH_GRADIENT) k_interact<SPH_GRADIENT, true><<<g, kThreads, 0, st>>>(a);
        else k_interact<SPH_FORCE, true><<<g, kThreads, 0, st>>>(a);
    } else {
        if (loop == SPH_DENSITY) k_interact<SPH_DENSITY, false><<<g, kThreads, 0, st>>>(a);
        else if (loop == SPH_GRADIENT) k_interact<SPH_GRADIENT, false><<<g, kThreads, 0, st>>>(a);
        else k_interact<SPH_FORCE, false><<<g, kThreads, 0, st>>>(a);
    }
    return launch_check("interaction kernel");
}

int sph_density(sph_tasks t, int bundle, const void *dev_buf_in, void *dev_buf_out,
                const sph_params *p, void *stream) {
    return interact(t, SPH_DENSITY, bundle, dev_buf_in, dev_buf_out, p, nullptr, stream);
}

int sph_gradient(sph_tasks t, int bundle, const void *dev_buf_in, void *dev_buf_out,
                 const sph_params *p, void *stream) {
    return interact(t, SPH_GRADIENT, bundle, dev_buf_in, dev_buf_out, p, nullptr, stream);
}

int sph_force(sph_tasks t, int bundle, const void *dev_buf_in, void *dev_buf_out,
              const sph_params *p, void *stream) {
    return interact(t, SPH_FORCE, bundle, dev_buf_in, dev_buf_out, p, nullptr, stream);
}

int sph_count_pairs(sph_tasks t, int loop, int bundle, const void *dev_buf_in,
                    const sph_params *p, unsigned long long *dev_count, void *stream) {
    if (int rc = check_loop(loop)) return rc;
    if (!dev_count) return fail(SPH_EINVAL, "NULL count");
    return interact(t, loop, bundle, dev_buf_in, nullptr, p, dev_count, stream);
}

int sph_unpack(sph_store s, sph_tasks t, int loop, int bundle, const void *dev_buf_out,
               void *stream) {
    StageRange range_(stage_name(ST_UNPACK, loop));
    if (int rc = check_store(s)) return rc;
    if (int rc = check_tasks(t, bundle)) return rc;
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_bundle_store(s, t)) return rc;
    if (!dev_buf_out || !aligned256(dev_buf_out))
        return fail(SPH_EINVAL, "result buffer must be a 256-byte aligned device pointer");
    UnpackArgs a{};
    const int64_t c0 = t->ucell_begin[bundle], nc = t->ucell_begin[bundle + 1] - c0;
    a.cells = t->d_ucells + c0;
    a.entries = t->d_entries + t->entry_begin[bundle];
    int nl;
    char *ol[4] = {nullptr, nullptr, nullptr, nullptr};
    lanes(loop, 1, t->bundle_slots[bundle], (char *)dev_buf_out, ol, &nl);
    a.lane[0] = ol[0];
    a.lane[1] = nl > 1 ? ol[1] : nullptr;
    int k = 0;
    if (loop == SPH_DENSITY) {
        a.dst[k++] = at(s, F_RHO, 0);
        a.dst[k++] = at(s, F_RHODH, 0);
        a.dst[k++] = at(s, F_WCOUNT, 0);
        a.dst[k++] = at(s, F_WCOUNTDH, 0);
        a.dst[k++] = at(s, F_DIVV, 0);
        for (int c = 0; c < 3; ++c) a.dst[k++] = at(s, F_ROTV, c);
    } else if (loop == SPH_GRADIENT) {
        a.dst[k++] = at(s, F_VSIGG, 0);
        a.dst[k++] = at(s, F_LAPU, 0);
    } else {
        for (int c = 0; c < 3; ++c) a.dst[k++] = at(s, F_A, c);
        a.dst[k++] = at(s, F_UDT, 0);
        a.dst[k++] = at(s, F_HDT, 0);
        a.dst[k++] = at(s, F_VSIG, 0);
    }
    if (nc == 0) return SPH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (loop == SPH_DENSITY) k_unpack<SPH_DENSITY><<<(unsigned)nc, 128, 0, st>>>(a);
    else if (loop == SPH_GRADIENT) k_unpack<SPH_GRADIENT><<<(unsigned)nc, 128, 0, st>>>(a);
    else k_unpack<SPH_FORCE><<<(unsigned)nc, 128, 0, st>>>(a);
    return launch_check("unpack");
}

int sph_ghost(sph_store s, int after_loop, const sph_params *p, void *stream) {
    if (int rc = check_store(s)) return rc;
    if (int rc = check_loop(after_loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (after_loop != SPH_DENSITY || s->n == 0) return SPH_OK;
    GhostArgs a{};
    const int roles[14][2] = {{F_MASS, 0}, {F_H, 0}, {F_U, 0}, {F_RHO, 0}, {F_RHODH, 0},
                              {F_WCOUNT, 0}, {F_DIVV, 0}, {F_ROTV, 0}, {F_ROTV, 1},
                              {F_ROTV, 2}, {F_FGRADH, 0}, {F_PRES, 0}, {F_CS, 0},
                              {F_BALS, 0}};
    for (int r = 0; r < 14; ++r) a.f[r] = at(s, roles[r][0], roles[r][1]);
    a.kernel_gamma = (float)p->kernel_gamma;
    a.gamma = (float)p->gamma;
    a.balsara_eps = (float)p->balsara_eps;
    k_ghost<<<grid_for(s->n, 256), 256, 0, (cudaStream_t)stream>>>(a, s->n);
    return launch_check("ghost");
}

int sph_offload_loop(sph_store s, sph_tasks t, int loop, void *dev_buf_in, void *dev_buf_out,
                     const sph_params *p, void *stream) {
    if (int rc = sph_init(s, loop, p, stream)) return rc;
    if (!t) return fail(SPH_EINVAL, "NULL tasks handle");
    const int nb = (int)t->bundle_slots.size();
    for (int b = 0; b < nb; ++b) {
        if (int rc = sph_pack(s, t, loop, b, dev_buf_in, stream)) return rc;
        if (int rc = interact(t, loop, b, dev_buf_in, dev_buf_out, p, nullptr, stream)) return rc;
        if (int rc = sph_unpack(s, t, loop, b, dev_buf_out, stream)) return rc;
    }
    return sph_ghost(s, loop, p, stream);
}

}  // extern "C"

// Scratch for sph_offload_loop_noalloc: one file-scope device array shared by
// every call on a device; its device address is looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SPH_NOALLOC_SCRATCH_BYTES];
static std::atomic<void *> g_noalloc_addr[64];

extern "C" {

int sph_offload_loop_noalloc(sph_store s, sph_tasks t, int loop, const sph_params *p,
                             void *stream) {
    if (int rc = check_store(s)) return rc;
    if (!t) return fail(SPH_EINVAL, "NULL tasks handle");
    if (int rc = check_loop(loop)) return rc;
    const size_t in_b = (sph_buffer_bytes(t, loop, 0) + 255) / 256 * 256;
    const size_t out_b = (sph_buffer_bytes(t, loop, 1) + 255) / 256 * 256;
    if (in_b + out_b > (size_t)SPH_NOALLOC_SCRATCH_BYTES)
        return fail(SPH_EUNSUPPORTED,
                    "noalloc: the largest bundle needs %zu + %zu bytes of buffers, more than "
                    "the %u-byte scratch array; rebuild the tasks with a smaller "
                    "bundle_max_slots",
                    in_b, out_b, (unsigned)SPH_NOALLOC_SCRATCH_BYTES);
    int dev = 0;
    if (int rc = cuda_check(cudaGetDevice(&dev), "noalloc: current device")) return rc;
    if (dev < 0 || dev >= 64) return fail(SPH_EUNSUPPORTED, "noalloc: device %d >= 64", dev);
    void *base = g_noalloc_addr[dev].load();
    if (!base) {
        if (int rc = cuda_check(cudaGetSymbolAddress(&base, g_noalloc_scratch),
                                "noalloc: scratch address"))
            return rc;
        g_noalloc_addr[dev].store(base);
    }
    char *buf_in = (char *)base;
    char *buf_out = buf_in + in_b;
    return sph_offload_loop(s, t, loop, buf_in, buf_out, p, stream);
}

int sph_sync(void *stream) {
    if (int rc = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "stream sync"))
        return rc;
    unsigned int w = 0;
    if (int rc = cuda_check(cudaMemcpyFromSymbol(&w, g_error_word, sizeof(w)), "error word"))
        return rc;
    if (w) {
        unsigned int z = 0;
        cudaMemcpyToSymbol(g_error_word, &z, sizeof(z));
        if (w & 8u)
            return fail(SPH_EUNSUPPORTED, "a particle's support exceeds what the batched plan "
                                          "was built for; rebuild the plan (word 0x%x)", w);
        if (w & 4u)
            return fail(SPH_ENOMEM, "neighbour list buffer too small: read "
                                    "sph_batch_list_status and grow it (word 0x%x)", w);
        if (w & 2u)
            return fail(SPH_ETIMEOUT, "a kernel's bounded wait for its copies ran out (word 0x%x)",
                        w);
        return fail(SPH_EBOUNDS, "a kernel reported an out-of-range index (word 0x%x)", w);
    }
    return SPH_OK;
}


int sph_store_create_host(int64_t n, int layout, uint64_t seed, void *host_mem, size_t bytes,
                          sph_store *out) {
    if (!out) return fail(SPH_EINVAL, "NULL out");
    *out = nullptr;
    if (n < 0 || n > INT32_MAX) return fail(SPH_EINVAL, "bad particle count %lld", (long long)n);
    Layout L;
    if (build_layout(layout, seed, n, &L) != SPH_OK)
        return fail(SPH_EINVAL, "bad layout %d", layout);
    const int64_t need = layout_bytes(L, n);
    if ((int64_t)bytes < need)
        return fail(SPH_EINVAL, "store needs %lld bytes, got %zu", (long long)need, bytes);
    if (need > 0 && (!host_mem || !aligned256(host_mem)))
        return fail(SPH_EINVAL, "store memory must be a 256-byte aligned host pointer");
    sph_store s = new (std::nothrow) sph_store_s;
    if (!s) return fail(SPH_ENOMEM, "store handle");
    s->n = n;
    s->layout = L;
    s->mem = (char *)host_mem;
    s->bytes = bytes;
    s->host = true;
    if (need > 0) memset(host_mem, 0, (size_t)need);
    *out = s;
    return SPH_OK;
}

int sph_store_import_host(sph_store s, const sph_fields *host_src, const int64_t *host_perm,
                          int nthreads) {
    if (int rc = check_host_store(s)) return rc;
    if (!host_src) return fail(SPH_EINVAL, "NULL fields");
    return host_copy_fields(s, host_src, host_perm, 1, nthreads);
}

int sph_store_export_host(sph_store s, const sph_fields *host_dst, const int64_t *host_perm,
                          int nthreads) {
    if (int rc = check_host_store(s)) return rc;
    if (!host_dst) return fail(SPH_EINVAL, "NULL fields");
    return host_copy_fields(s, host_dst, host_perm, 0, nthreads);
}

static int check_host_bundle(sph_store s, sph_tasks t, int loop, int bundle) {
    if (int rc = check_host_store(s)) return rc;
    if (!t) return fail(SPH_EINVAL, "NULL tasks handle");
    if (int rc = check_loop(loop)) return rc;
    if (bundle < 0 || bundle >= (int64_t)t->bundle_slots.size())
        return fail(SPH_EINVAL, "bundle %d out of range", bundle);
    if (s->n != t->n) return fail(SPH_EINVAL, "store and tasks disagree on particle count");
    return SPH_OK;
}

int sph_pack_host(sph_store s, sph_tasks t, int loop, int bundle, void *host_buf_in,
                  int nthreads) {
    if (int rc = check_host_bundle(s, t, loop, bundle)) return rc;
    if (!host_buf_in || !aligned256(host_buf_in))
        return fail(SPH_EINVAL, "pack buffer must be a 256-byte aligned host pointer");
    return host_pack(s, t, loop, bundle, (char *)host_buf_in, nthreads);
}

int sph_unpack_host(sph_store s, sph_tasks t, int loop, int bundle, const void *host_buf_out,
                    int nthreads) {
    if (int rc = check_host_bundle(s, t, loop, bundle)) return rc;
    if (!host_buf_out || !aligned256(host_buf_out))
        return fail(SPH_EINVAL, "result buffer must be a 256-byte aligned host pointer");
    return host_unpack(s, t, loop, bundle, (const char *)host_buf_out, nthreads);
}

int sph_pack_host_fission(sph_store s, sph_tasks t, int loop, int bundle, void *host_buf_in,
                          int fission, int nthreads) {
    if (int rc = check_host_bundle(s, t, loop, bundle)) return rc;
    if (fission < SPH_FISSION_NONE || fission > SPH_FISSION_BY_STRUCT_AND_TYPE)
        return fail(SPH_EINVAL, "unknown loop-fission variant %d", fission);
    if (!host_buf_in || !aligned256(host_buf_in))
        return fail(SPH_EINVAL, "pack buffer must be a 256-byte aligned host pointer");
    return host_pack_fission(s, t, loop, bundle, (char *)host_buf_in, fission, nthreads);
}

int sph_unpack_host_fission(sph_store s, sph_tasks t, int loop, int bundle,
                            const void *host_buf_out, int fission, int nthreads) {
    if (int rc = check_host_bundle(s, t, loop, bundle)) return rc;
    if (fission < SPH_FISSION_NONE || fission > SPH_FISSION_BY_STRUCT_AND_TYPE)
        return fail(SPH_EINVAL, "unknown loop-fission variant %d", fission);
    if (!host_buf_out || !aligned256(host_buf_out))
        return fail(SPH_EINVAL, "result buffer must be a 256-byte aligned host pointer");
    return host_unpack_fission(s, t, loop, bundle, (const char *)host_buf_out, fission,
                               nthreads);
}

int sph_init_host(sph_store s, int loop, const sph_params *p, int nthreads) {
    if (int rc = check_host_store(s)) return rc;
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    return host_init(s, loop, p->active_bin, nthreads);
}

int sph_ghost_host(sph_store s, int after_loop, const sph_params *p, int nthreads) {
    if (int rc = check_host_store(s)) return rc;
    if (int rc = check_loop(after_loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (after_loop != SPH_DENSITY) return SPH_OK;
    return host_ghost(s, (float)p->kernel_gamma, (float)p->gamma, (float)p->balsara_eps, nthreads);
}

}  // extern "C"

namespace sph {

static double host_now() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

// The host-staged cycle of one loop; with `stats`, every stage is timed: the
// host pack, unpack and waits on the host clock, the copies and the kernel
// of each bundle with CUDA events on its stream.
static int offload_loop_host(sph_store s, sph_tasks t, int loop, void *const host_in[2],
                             void *const host_out[2], void *const dev_in[2],
                             void *const dev_out[2], const sph_params *p,
                             void *const streams[2], int nthreads, sph_staged_stats *stats) {
    if (int rc = check_host_store(s)) return rc;
    if (!t) return fail(SPH_EINVAL, "NULL tasks handle");
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (!host_in || !host_out || !dev_in || !dev_out || !streams)
        return fail(SPH_EINVAL, "NULL buffer or stream array");
    for (int k = 0; k < 2; ++k)
        if (!aligned256(host_in[k]) || !aligned256(host_out[k]) || !aligned256(dev_in[k]) ||
            !aligned256(dev_out[k]) || !host_in[k] || !host_out[k] || !dev_in[k] || !dev_out[k])
            return fail(SPH_EINVAL, "buffers must be non-NULL and 256-byte aligned");
    const double t_start = host_now();
    double t_pack = 0.0, t_unpack = 0.0, t_wait = 0.0;
    int64_t h2d_bytes = 0, d2h_bytes = 0;
    if (int rc = host_init(s, loop, p->active_bin, nthreads)) return rc;
    const int nb = (int)t->bundle_slots.size();
    cudaStream_t st[2] = {(cudaStream_t)streams[0], (cudaStream_t)streams[1]};
    cudaEvent_t done[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> tev;   // per bundle: before H2D, after H2D, after kernel, after D2H
    int rc = SPH_OK;
    for (int k = 0; k < 2 && rc == SPH_OK; ++k)
        rc = cuda_check(cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming), "event");
    if (stats && rc == SPH_OK) {
        tev.assign(4 * (size_t)nb, nullptr);
        for (size_t e = 0; e < tev.size() && rc == SPH_OK; ++e)
            rc = cuda_check(cudaEventCreate(&tev[e]), "timing event");
    }
    auto mark = [&](int b, int q, cudaStream_t s_) -> int {
        return stats ? cuda_check(cudaEventRecord(tev[4 * (size_t)b + q], s_), "event record")
                     : SPH_OK;
    };
    for (int b = 0; b < nb && rc == SPH_OK; ++b) {
        const int k = b & 1;
        int64_t off[16];
        const size_t in_b = (size_t)lane_offsets(loop, 0, t->bundle_slots[b], off);
        const size_t out_b = (size_t)lane_offsets(loop, 1, t->bundle_slots[b], off);
        // buffers k were last used by bundle b-2, whose results were unpacked
        // after its event completed in the previous iteration
        double t0 = host_now();
        if ((rc = sph_pack_host(s, t, loop, b, host_in[k], nthreads))) break;
        t_pack += host_now() - t0;
        if ((rc = mark(b, 0, st[k]))) break;
        if ((rc = cuda_check(cudaMemcpyAsync(dev_in[k], host_in[k], in_b,
                                             cudaMemcpyHostToDevice, st[k]), "H2D")))
            break;
        if ((rc = mark(b, 1, st[k]))) break;
        if ((rc = interact(t, loop, b, dev_in[k], dev_out[k], p, nullptr, st[k]))) break;
        if ((rc = mark(b, 2, st[k]))) break;
        if ((rc = cuda_check(cudaMemcpyAsync(host_out[k], dev_out[k], out_b,
                                             cudaMemcpyDeviceToHost, st[k]), "D2H")))
            break;
        if ((rc = mark(b, 3, st[k]))) break;
        h2d_bytes += (int64_t)in_b;
        d2h_bytes += (int64_t)out_b;
        if ((rc = cuda_check(cudaEventRecord(done[k], st[k]), "event record"))) break;
        if (b >= 1) {
            t0 = host_now();
            if ((rc = cuda_check(cudaEventSynchronize(done[k ^ 1]), "event wait"))) break;
            const double t1 = host_now();
            t_wait += t1 - t0;
            if ((rc = sph_unpack_host(s, t, loop, b - 1, host_out[k ^ 1], nthreads))) break;
            t_unpack += host_now() - t1;
        }
    }
    if (rc == SPH_OK && nb > 0) {
        const int k = (nb - 1) & 1;
        double t0 = host_now();
        rc = cuda_check(cudaEventSynchronize(done[k]), "event wait");
        const double t1 = host_now();
        t_wait += t1 - t0;
        if (rc == SPH_OK) rc = sph_unpack_host(s, t, loop, nb - 1, host_out[k], nthreads);
        t_unpack += host_now() - t1;
    }
    if (rc != SPH_OK) {
        cudaStreamSynchronize(st[0]);
        cudaStreamSynchronize(st[1]);
    }
    for (int k = 0; k < 2; ++k)
        if (done[k]) cudaEventDestroy(done[k]);
    if (rc == SPH_OK && loop == SPH_DENSITY) {
        const double t0 = host_now();
        rc = sph_ghost_host(s, SPH_DENSITY, p, nthreads);
        t_unpack += host_now() - t0;
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        for (int b = 0; b < nb && rc == SPH_OK; ++b) {
            float ms[3] = {0.f, 0.f, 0.f};
            for (int q = 0; q < 3 && rc == SPH_OK; ++q)
                rc = cuda_check(cudaEventElapsedTime(&ms[q], tev[4 * (size_t)b + q],
                                                     tev[4 * (size_t)b + q + 1]),
                                "elapsed time");
            stats->h2d_ms += ms[0];
            stats->kernel_ms += ms[1];
            stats->d2h_ms += ms[2];
        }
        for (cudaEvent_t e : tev)
            if (e) cudaEventDestroy(e);
        stats->wall_s = host_now() - t_start;
        stats->host_pack_s = t_pack;
        stats->host_unpack_s = t_unpack;
        stats->host_wait_s = t_wait;
        stats->h2d_bytes = h2d_bytes;
        stats->d2h_bytes = d2h_bytes;
        stats->bundles = nb;
    }
    return rc;
}

}  // namespace sph

extern "C" {

int sph_offload_loop_host(sph_store s, sph_tasks t, int loop, void *const host_in[2],
                          void *const host_out[2], void *const dev_in[2], void *const dev_out[2],
                          const sph_params *p, void *const streams[2], int nthreads) {
    return offload_loop_host(s, t, loop, host_in, host_out, dev_in, dev_out, p, streams,
                             nthreads, nullptr);
}

int sph_offload_loop_host_stats(sph_store s, sph_tasks t, int loop, void *const host_in[2],
                                void *const host_out[2], void *const dev_in[2],
                                void *const dev_out[2], const sph_params *p,
                                void *const streams[2], int nthreads, sph_staged_stats *stats) {
    if (!stats) return fail(SPH_EINVAL, "NULL stats");
    return offload_loop_host(s, t, loop, host_in, host_out, dev_in, dev_out, p, streams,
                             nthreads, stats);
}

// ---- batched (cell-dedup) pipeline ---------------------------------------
static int check_batch(sph_batch b, int bundle) {
    if (!b) return fail(SPH_EINVAL, "NULL batch handle");
    if (bundle < 0 || bundle >= (int64_t)b->bundles.size())
        return fail(SPH_EINVAL, "bundle %d out of range", bundle);
    return SPH_OK;
}

static void batch_free(sph_batch b) {
    if (b->d_naux) cudaFree(b->d_naux);
    if (b->d_mbase) cudaFree(b->d_mbase);
    if (b->d_rev) cudaFree(b->d_rev);
    if (b->d_rev_start) cudaFree(b->d_rev_start);
    b->d_naux = nullptr;
    b->d_mbase = nullptr;
    b->d_rev = nullptr;
    b->d_rev_start = nullptr;
    if (b->d_cells) cudaFree(b->d_cells);
    if (b->d_targets) cudaFree(b->d_targets);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_nbrs) cudaFree(b->d_nbrs);
    if (b->d_counter) cudaFree(b->d_counter);
    b->d_nbrs = nullptr;
    b->d_cells = nullptr;
    b->d_targets = nullptr;
    b->d_items = nullptr;
    b->d_counter = nullptr;
}

// Copy a built plan to the current device; frees and deletes it on failure.
static int batch_upload(sph_batch b, int rc, sph_batch *out) {
    auto up = [&](void **dst, const void *src, size_t bytes, const char *what) -> int {
        return upload_meta(dst, src, bytes, what);
    };
    if (rc == SPH_OK &&
        ((rc = up((void **)&b->d_cells, b->cells.data(), b->cells.size() * sizeof(BCellDev),
                  "batch cells")) ||
         (rc = up((void **)&b->d_targets, b->targets.data(),
                  b->targets.size() * sizeof(BTargetDev), "batch targets")) ||
         (rc = up((void **)&b->d_nbrs, b->nbrs.data(), b->nbrs.size() * sizeof(BNbrDev),
                  "batch neighbour entries")) ||
         (rc = up((void **)&b->d_items, b->items.data(), b->items.size() * sizeof(BItemDev),
                  "batch items")) ||
         (rc = up((void **)&b->d_counter, nullptr,
                  (b->bundles.size() + 1) * sizeof(unsigned int), "batch counters")) ||
         (b->sym && ((rc = up((void **)&b->d_naux, b->naux.data(),
                              b->naux.size() * sizeof(int32_t), "symmetric list entries")) ||
                     (rc = up((void **)&b->d_mbase, b->mbase.data(),
                              b->mbase.size() * sizeof(long long), "symmetric list masks")) ||
                     (rc = up((void **)&b->d_rev, b->rev.data(),
                              b->rev.size() * sizeof(RevEntDev), "symmetric list neighbours")) ||
                     (rc = up((void **)&b->d_rev_start, b->rev_start.data(),
                              b->rev_start.size() * sizeof(int32_t),
                              "symmetric list neighbour starts")))))) {
    }
    if (rc) {
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return SPH_OK;
}

int sph_batch_build(sph_tasks t, const sph_batch_params *bp, sph_batch *out) {
    if (!out) return fail(SPH_EINVAL, "NULL out");
    *out = nullptr;
    if (!t || !bp) return fail(SPH_EINVAL, "NULL tasks or params");
    if (bp->reserved != 0) return fail(SPH_EINVAL, "batch params: reserved must be 0");
    sph_batch b = new (std::nothrow) sph_batch_s;
    if (!b) return fail(SPH_ENOMEM, "batch handle");
    int rc;
    try {
        rc = build_batch(t, bp, b);
    } catch (const std::bad_alloc &) {
        rc = fail(SPH_ENOMEM, "batch_build: host allocation failed");
    }
    return batch_upload(b, rc, out);
}

int sph_batch_build_tree(int64_t n, const double *host_x, const float *host_h,
                         const sph_tree_params *tp, const sph_batch_params *bp,
                         int64_t *host_perm_out, sph_batch *out) {
    if (!out) return fail(SPH_EINVAL, "NULL out");
    *out = nullptr;
    if (!tp || !bp) return fail(SPH_EINVAL, "NULL tree or batch params");
    if (bp->reserved != 0) return fail(SPH_EINVAL, "batch params: reserved must be 0");
    sph_batch b = new (std::nothrow) sph_batch_s;
    if (!b) return fail(SPH_ENOMEM, "batch handle");
    int rc;
    try {
        rc = build_batch_tree(n, host_x, host_h, tp, bp, host_perm_out, b);
    } catch (const std::bad_alloc &) {
        rc = fail(SPH_ENOMEM, "batch_build_tree: host allocation failed");
    }
    return batch_upload(b, rc, out);
}

int sph_tree_plan(int64_t n, const double *host_x, const float *host_h,
                  const sph_tree_params *tp, int64_t *host_perm_out,
                  int64_t *host_leaf_start, int64_t *nleaf_out, int64_t *host_nb_start,
                  int32_t *host_nb, int64_t nb_cap, int64_t *nnb_out) {
    try {
        return tree_plan_host(n, host_x, host_h, tp, host_perm_out, host_leaf_start, nleaf_out,
                              host_nb_start, host_nb, nb_cap, nnb_out);
    } catch (const std::bad_alloc &) {
        return fail(SPH_ENOMEM, "tree_plan: host allocation failed");
    }
}

int sph_batch_list_fixed(sph_batch b) {
    if (!b) return -fail(SPH_EINVAL, "NULL batch handle");
    return b->fixed_build ? 1 : 0;
}

int sph_batch_list_symmetric(sph_batch b, int enable) {
    if (!b) return -fail(SPH_EINVAL, "NULL batch handle");
    if (enable >= 0) b->sym_on = enable != 0;
    return b->sym && b->sym_on ? 1 : 0;
}

int sph_batch_cells(sph_batch b, int bundle, int32_t *cells, int64_t *ncells) {
    if (int rc = check_batch(b, bundle)) return rc;
    if (!ncells) return fail(SPH_EINVAL, "NULL argument");
    const BatchBundle &bb = b->bundles[bundle];
    *ncells = bb.ncells;
    if (!cells) return SPH_OK;
    for (int64_t c = 0; c < bb.ncells; ++c) {
        const BCellDev &cd = b->cells[bb.cell0 + c];
        cells[3 * c + 0] = cd.p0;
        cells[3 * c + 1] = cd.n;
        cells[3 * c + 2] = cd.slot;
    }
    return SPH_OK;
}

int sph_batch_plan_info(sph_batch b, int64_t info[4]) {
    if (!b || !info) return fail(SPH_EINVAL, "NULL argument");
    info[0] = b->kind;
    info[1] = b->plan_cells;
    info[2] = b->plan_max_cell;
    info[3] = b->plan_nbrs;
    return SPH_OK;
}

int sph_batch_info(sph_batch b, int64_t info[6]) {
    if (!b || !info) return fail(SPH_EINVAL, "NULL argument");
    info[0] = (int64_t)b->bundles.size();
    info[1] = b->max_slots;
    info[2] = (int64_t)b->items.size();
    info[3] = b->threads;
    info[4] = b->max_targets;
    info[5] = (int64_t)b->cells.size();
    return SPH_OK;
}

static int64_t batch_max_cells(sph_batch b) {
    int64_t m = 0;
    for (const BatchBundle &bb : b->bundles) m = bb.ncells > m ? bb.ncells : m;
    return m;
}

size_t sph_batch_buffer_bytes(sph_batch b, int loop, int in_or_out) {
    if (!b || loop < SPH_DENSITY || loop > SPH_FORCE || (in_or_out != 0 && in_or_out != 1))
        return 0;
    const int64_t S = b->max_slots, C = batch_max_cells(b);
    if (in_or_out == 1) return (size_t)bout_bytes(loop, S);
    if (loop == SPH_DENSITY) return (size_t)BLayout<SPH_DENSITY>::bytes(S, C);
    if (loop == SPH_GRADIENT) return (size_t)BLayout<SPH_GRADIENT>::bytes(S, C);
    return (size_t)BLayout<SPH_FORCE>::bytes(S, C);
}

static int batch_pack(sph_store s, sph_batch b, int loop, int bundle, void *dev_buf_in,
                      const sph_params *p, void *stream, bool compact);

int sph_batch_pack(sph_store s, sph_batch b, int loop, int bundle, void *dev_buf_in,
                   const sph_params *p, void *stream) {
    return batch_pack(s, b, loop, bundle, dev_buf_in, p, stream, false);
}

int sph_batch_pack_list(sph_store s, sph_batch b, int loop, int bundle, void *dev_buf_in,
                        const sph_params *p, void *stream) {
    return batch_pack(s, b, loop, bundle, dev_buf_in, p, stream, true);
}

static int batch_pack(sph_store s, sph_batch b, int loop, int bundle, void *dev_buf_in,
                      const sph_params *p, void *stream, bool compact) {
    StageRange range_(stage_name(ST_PACK, loop));
    if (int rc = check_store(s)) return rc;
    if (int rc = check_batch(b, bundle)) return rc;
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (!dev_buf_in || !aligned256(dev_buf_in))
        return fail(SPH_EINVAL, "pack buffer must be a 256-byte aligned device pointer");
    const BatchBundle &bb = b->bundles[bundle];
    BPackArgs a{};
    a.cells = b->d_cells + bb.cell0;
    a.buf = (char *)dev_buf_in;
    a.S = bb.slots;
    for (int d = 0; d < 3; ++d) a.fx_scale[d] = 4294967296.0 / b->box[d];
    const int roles[R_NUM][2] = {{F_X, 0}, {F_X, 1}, {F_X, 2}, {F_V, 0}, {F_V, 1},
                                 {F_V, 2}, {F_MASS, 0}, {F_H, 0}, {F_U, 0}, {F_RHO, 0},
                                 {F_FGRADH, 0}, {F_BALS, 0}, {F_AVISC, 0}, {F_ADIFF, 0},
                                 {F_TBIN, 0}};
    for (int r = 0; r < R_NUM; ++r) a.src[r] = at_view(s, roles[r][0], roles[r][1], loop);
    a.kernel_gamma = (float)p->kernel_gamma;
    a.gamma = (float)p->gamma;
    double bmax = b->box[0] > b->box[1] ? b->box[0] : b->box[1];
    bmax = bmax > b->box[2] ? bmax : b->box[2];
    a.delta = (float)(4e-6 * bmax);
    if (bb.ncells == 0) return SPH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    a.ncells = (int)bb.ncells;
    a.min_n = kWPack + 1;
    // cells of up to kWPack particles: one warp each (k_bpack_w); larger ones:
    // one 64-thread CTA each (k_bpack), launched only when the plan has them
    const unsigned gw = (unsigned)((bb.ncells + 3) / 4), g = (unsigned)bb.ncells;
    const bool big = b->plan_max_cell > kWPack;
    // the list loops' density pack writes only the fixed-point lanes where the
    // list build reads nothing else (plans on the fixed-point path)
    if (loop == SPH_DENSITY && compact && b->fixed_build) {
        k_bpack_w<SPH_DENSITY, true><<<gw, 128, 0, st>>>(a);
        if (big) k_bpack<SPH_DENSITY, true><<<g, 64, 0, st>>>(a);
    } else if (loop == SPH_DENSITY) {
        k_bpack_w<SPH_DENSITY><<<gw, 128, 0, st>>>(a);
        if (big) k_bpack<SPH_DENSITY><<<g, 64, 0, st>>>(a);
    } else if (loop == SPH_GRADIENT && compact) {
        k_bpack_w<SPH_GRADIENT, true><<<gw, 128, 0, st>>>(a);
        if (big) k_bpack<SPH_GRADIENT, true><<<g, 64, 0, st>>>(a);
    } else if (loop == SPH_GRADIENT) {
        k_bpack_w<SPH_GRADIENT><<<gw, 128, 0, st>>>(a);
        if (big) k_bpack<SPH_GRADIENT><<<g, 64, 0, st>>>(a);
    } else if (compact) {
        k_bpack_w<SPH_FORCE, true><<<gw, 128, 0, st>>>(a);
        if (big) k_bpack<SPH_FORCE, true><<<g, 64, 0, st>>>(a);
    } else {
        k_bpack_w<SPH_FORCE><<<gw, 128, 0, st>>>(a);
        if (big) k_bpack<SPH_FORCE><<<g, 64, 0, st>>>(a);
    }
    return launch_check("batch pack");
}

static BInteractArgs interact_args(sph_batch b, int bundle, const void *dev_buf_in,
                                   void *dev_buf_out, const sph_params *p) {
    const BatchBundle &bb = b->bundles[bundle];
    BInteractArgs a{};
    a.naux = b->d_naux;
    a.mbase = b->d_mbase;
    a.rev = b->d_rev;
    a.rev_start = b->d_rev_start;
    a.sym_words = b->sym_words;
    a.cells = b->d_cells + bb.cell0;
    a.targets = b->d_targets + bb.target0;
    a.nbrs = b->d_nbrs;
    a.items = b->d_items + bb.item0;
    a.counter = b->d_counter + bundle;
    a.nitems = (int)bb.nitems;
    a.in = (const char *)dev_buf_in;
    a.out = (char *)dev_buf_out;
    a.S = bb.slots;
    a.kernel_gamma = (float)p->kernel_gamma;
    a.gamma = (float)p->gamma;
    a.beta = (float)p->beta_visc;
    double bmax = b->box[0] > b->box[1] ? b->box[0] : b->box[1];
    bmax = bmax > b->box[2] ? bmax : b->box[2];
    a.delta = (float)(4e-6 * bmax);
    for (int d = 0; d < 3; ++d) {
        a.shift_hi[d] = (float)b->box[d];
        a.shift_lo[d] = (float)(b->box[d] - (double)a.shift_hi[d]);
        a.half[d] = (float)(0.5 * b->box[d]);
        a.fx_unit[d] = (float)(b->box[d] / 4294967296.0);
    }
    a.active_bin = p->active_bin;
    a.pa.beta = a.beta;
    a.pa.kernel_gamma = a.kernel_gamma;
    a.pa.gamma = a.gamma;
    a.pa.delta = a.delta;
    a.pa.active_bin = a.active_bin;
    return a;
}

int sph_batch_interact(sph_batch b, int loop, int bundle, const void *dev_buf_in,
                       void *dev_buf_out, const sph_params *p, void *stream) {
    StageRange range_(stage_name(ST_INTERACT, loop));
    if (int rc = check_batch(b, bundle)) return rc;
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_buf_out || !aligned256(dev_buf_out))
        return fail(SPH_EINVAL, "buffers must be 256-byte aligned device pointers");
    const BatchBundle &bb = b->bundles[bundle];
    BInteractArgs a = interact_args(b, bundle, dev_buf_in, dev_buf_out, p);
    cudaStream_t st = (cudaStream_t)stream;
    if (bb.nitems == 0) return SPH_OK;
    if (int rc = cuda_check(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st),
                            "reset work queue"))
        return rc;
    if (loop == SPH_DENSITY) return dispatch_binteract<SPH_DENSITY>(b->threads, a, st);
    if (loop == SPH_GRADIENT) return dispatch_binteract<SPH_GRADIENT>(b->threads, a, st);
    return dispatch_binteract<SPH_FORCE>(b->threads, a, st);
}

static int batch_unpack(sph_store s, sph_batch b, int loop, int bundle, const void *dev_buf_out,
                        const void *dev_buf_in, bool write, bool ghost, const sph_params *p,
                        void *stream) {
    StageRange range_(stage_name(ST_UNPACK, loop));
    if (int rc = check_store(s)) return rc;
    if (int rc = check_batch(b, bundle)) return rc;
    if (int rc = check_loop(loop)) return rc;
    if (!dev_buf_in || !dev_buf_out) return fail(SPH_EINVAL, "NULL buffer");
    const BatchBundle &bb = b->bundles[bundle];
    BUnpackArgs a{};
    a.cells = b->d_cells + bb.cell0;
    a.targets = b->d_targets + bb.target0;
    a.out = (const char *)dev_buf_out;
    const int64_t S = bb.slots;
    int64_t perm_off = loop == SPH_DENSITY ? BLayout<SPH_DENSITY>::perm(S)
                       : loop == SPH_GRADIENT ? BLayout<SPH_GRADIENT>::perm(S)
                                              : BLayout<SPH_FORCE>::perm(S);
    a.perm = reinterpret_cast<const int32_t *>((const char *)dev_buf_in + perm_off);
    a.tb = reinterpret_cast<const int8_t *>((const char *)dev_buf_in + BLayout<SPH_FORCE>::tb(S));
    a.active_bin = p ? p->active_bin : 0;
    a.S = S;
    ghost = ghost && loop == SPH_DENSITY;
    if (ghost) {
        a.gin[0] = at(s, F_MASS, 0);
        a.gin[1] = at(s, F_H, 0);
        a.gin[2] = at(s, F_U, 0);
        a.gout[0] = at(s, F_FGRADH, 0);
        a.gout[1] = at(s, F_PRES, 0);
        a.gout[2] = at(s, F_CS, 0);
        a.gout[3] = at(s, F_BALS, 0);
        a.kernel_gamma = (float)p->kernel_gamma;
        a.gamma = (float)p->gamma;
        a.balsara_eps = (float)p->balsara_eps;
    }
    int k = 0;
    if (loop == SPH_DENSITY) {
        for (int f : {F_RHO, F_RHODH, F_WCOUNT, F_WCOUNTDH, F_DIVV}) a.dst[k++] = at(s, f, 0);
        for (int c = 0; c < 3; ++c) a.dst[k++] = at(s, F_ROTV, c);
    } else if (loop == SPH_GRADIENT) {
        a.dst[k++] = at(s, F_VSIGG, 0);
        a.dst[k++] = at(s, F_LAPU, 0);
    } else {
        for (int c = 0; c < 3; ++c) a.dst[k++] = at(s, F_A, c);
        for (int f : {F_UDT, F_HDT, F_VSIG}) a.dst[k++] = at(s, f, 0);
    }
    if (bb.ntargets == 0) return SPH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned g = (unsigned)bb.ntargets;
    if (ghost) {
        // rho_dh .. rot_v as seven consecutive words of one record, and small
        // enough cells: the form that writes them in store order
        bool run7 = b->plan_max_cell <= kUnpC;
        for (int j = 2; j < 8 && run7; ++j)
            run7 = a.dst[j].stride == a.dst[1].stride && a.dst[j].ptr == a.dst[1].ptr + 4 * (j - 1);
        if (run7) k_bunpack_dg<<<g, 64, 0, st>>>(a);
        else k_bunpack<SPH_DENSITY, true, true><<<g, 64, 0, st>>>(a);
    } else if (write) {
        if (loop == SPH_DENSITY) k_bunpack<SPH_DENSITY, true><<<g, 64, 0, st>>>(a);
        else if (loop == SPH_GRADIENT) k_bunpack<SPH_GRADIENT, true><<<g, 64, 0, st>>>(a);
        else k_bunpack<SPH_FORCE, true><<<g, 64, 0, st>>>(a);
    } else {
        if (loop == SPH_DENSITY) k_bunpack<SPH_DENSITY><<<g, 64, 0, st>>>(a);
        else if (loop == SPH_GRADIENT) k_bunpack<SPH_GRADIENT><<<g, 64, 0, st>>>(a);
        else k_bunpack<SPH_FORCE><<<g, 64, 0, st>>>(a);
    }
    return launch_check("batch unpack");
}

int sph_batch_unpack(sph_store s, sph_batch b, int loop, int bundle, const void *dev_buf_out,
                     const void *dev_buf_in, void *stream) {
    return batch_unpack(s, b, loop, bundle, dev_buf_out, dev_buf_in, false, false, nullptr,
                        stream);
}

int sph_batch_unpack_write(sph_store s, sph_batch b, int loop, int bundle,
                           const void *dev_buf_out, const void *dev_buf_in, const sph_params *p,
                           int with_ghost, void *stream) {
    if (int rc = check_params(p)) return rc;
    return batch_unpack(s, b, loop, bundle, dev_buf_out, dev_buf_in, true, with_ghost != 0, p,
                        stream);
}

int sph_batch_offload_loop(sph_store s, sph_batch b, int loop, void *dev_buf_in,
                           void *dev_buf_out, const sph_params *p, void *stream) {
    if (int rc = check_store(s)) return rc;
    if (!b) return fail(SPH_EINVAL, "NULL batch handle");
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    for (int k = 0; k < (int)b->bundles.size(); ++k) {
        if (int rc = sph_batch_pack(s, b, loop, k, dev_buf_in, p, stream)) return rc;
        if (int rc = sph_batch_interact(b, loop, k, dev_buf_in, dev_buf_out, p, stream)) return rc;
        if (int rc = sph_batch_unpack_write(s, b, loop, k, dev_buf_out, dev_buf_in, p, 1,
                                            stream))
            return rc;
    }
    return SPH_OK;
}

int sph_batch_destroy(sph_batch b) {
    if (!b) return SPH_OK;
    batch_free(b);
    delete b;
    return SPH_OK;
}

size_t sph_batch_buffer_bytes_fp64(sph_batch b, int in_or_out) {
    if (!b || (in_or_out != 0 && in_or_out != 1)) return 0;
    if (in_or_out == 0) return (size_t)D64Layout::bytes(b->max_slots);
    return (size_t)D64Layout::out_bytes(SPH_DENSITY, b->max_slots);
}

int sph_batch_offload_loop_fp64(sph_store s, sph_batch b, int loop, void *dev_buf_in,
                                void *dev_buf_out, const sph_params *p, void *stream) {
    if (int rc = check_store(s)) return rc;
    if (!b) return fail(SPH_EINVAL, "NULL batch handle");
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_buf_out || !aligned256(dev_buf_out))
        return fail(SPH_EINVAL, "buffers must be 256-byte aligned device pointers");
    if (int rc = sph_init(s, loop, p, stream)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int roles[R_NUM][2] = {{F_X, 0}, {F_X, 1}, {F_X, 2}, {F_V, 0}, {F_V, 1},
                                 {F_V, 2}, {F_MASS, 0}, {F_H, 0}, {F_U, 0}, {F_RHO, 0},
                                 {F_FGRADH, 0}, {F_BALS, 0}, {F_AVISC, 0}, {F_ADIFF, 0},
                                 {F_TBIN, 0}};
    for (int k = 0; k < (int)b->bundles.size(); ++k) {
        const BatchBundle &bb = b->bundles[k];
        if (bb.ncells == 0 || bb.ntargets == 0) continue;
        D64PackArgs pa{};
        pa.cells = b->d_cells + bb.cell0;
        pa.buf = (char *)dev_buf_in;
        pa.S = bb.slots;
        for (int r = 0; r < R_NUM; ++r) pa.src[r] = at(s, roles[r][0], roles[r][1]);
        pa.kernel_gamma = p->kernel_gamma;
        k_pack64<<<(unsigned)bb.ncells, 128, 0, st>>>(pa);
        if (int rc = launch_check("fp64 pack")) return rc;
        D64Args ia{};
        ia.cells = b->d_cells + bb.cell0;
        ia.targets = b->d_targets + bb.target0;
        ia.nbrs = b->d_nbrs;
        ia.in = (const char *)dev_buf_in;
        ia.out = (char *)dev_buf_out;
        ia.S = bb.slots;
        ia.gamma = p->gamma;
        ia.beta = p->beta_visc;
        for (int d = 0; d < 3; ++d) ia.box[d] = b->box[d];
        ia.active_bin = p->active_bin;
        const unsigned g = (unsigned)bb.ntargets;
        if (loop == SPH_DENSITY) k_interact64<SPH_DENSITY><<<g, 128, 0, st>>>(ia);
        else if (loop == SPH_GRADIENT) k_interact64<SPH_GRADIENT><<<g, 128, 0, st>>>(ia);
        else k_interact64<SPH_FORCE><<<g, 128, 0, st>>>(ia);
        if (int rc = launch_check("fp64 interaction kernel")) return rc;
        D64UnpackArgs ua{};
        ua.cells = b->d_cells + bb.cell0;
        ua.targets = b->d_targets + bb.target0;
        ua.out = (const double *)dev_buf_out;
        ua.perm = reinterpret_cast<const int32_t *>((const char *)dev_buf_in +
                                                    D64Layout::perm(bb.slots));
        int q = 0;
        if (loop == SPH_DENSITY) {
            for (int f : {F_RHO, F_RHODH, F_WCOUNT, F_WCOUNTDH, F_DIVV}) ua.dst[q++] = at(s, f, 0);
            for (int c = 0; c < 3; ++c) ua.dst[q++] = at(s, F_ROTV, c);
        } else if (loop == SPH_GRADIENT) {
            ua.dst[q++] = at(s, F_VSIGG, 0);
            ua.dst[q++] = at(s, F_LAPU, 0);
        } else {
            for (int c = 0; c < 3; ++c) ua.dst[q++] = at(s, F_A, c);
            for (int f : {F_UDT, F_HDT, F_VSIG}) ua.dst[q++] = at(s, f, 0);
        }
        if (loop == SPH_DENSITY) k_unpack64<SPH_DENSITY><<<g, 128, 0, st>>>(ua);
        else if (loop == SPH_GRADIENT) k_unpack64<SPH_GRADIENT><<<g, 128, 0, st>>>(ua);
        else k_unpack64<SPH_FORCE><<<g, 128, 0, st>>>(ua);
        if (int rc = launch_check("fp64 unpack")) return rc;
    }
    if (loop != SPH_DENSITY || s->n == 0) return SPH_OK;
    GhostArgs ga{};
    const int groles[14][2] = {{F_MASS, 0}, {F_H, 0}, {F_U, 0}, {F_RHO, 0}, {F_RHODH, 0},
                               {F_WCOUNT, 0}, {F_DIVV, 0}, {F_ROTV, 0}, {F_ROTV, 1},
                               {F_ROTV, 2}, {F_FGRADH, 0}, {F_PRES, 0}, {F_CS, 0},
                               {F_BALS, 0}};
    for (int r = 0; r < 14; ++r) ga.f[r] = at(s, groles[r][0], groles[r][1]);
    k_ghost64<<<grid_for(s->n, 256), 256, 0, st>>>(ga, s->n, p->kernel_gamma, p->gamma,
                                                    p->balsara_eps);
    return launch_check("fp64 ghost");
}

int sph_batch_count_pairs(sph_store s, sph_batch b, int loop, void *dev_buf_in,
                          const sph_params *p, unsigned long long *dev_count, void *stream) {
    if (int rc = check_store(s)) return rc;
    if (!b) return fail(SPH_EINVAL, "NULL batch handle");
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_count)
        return fail(SPH_EINVAL, "buffer must be a 256-byte aligned device pointer; count non-NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int roles[R_NUM][2] = {{F_X, 0}, {F_X, 1}, {F_X, 2}, {F_V, 0}, {F_V, 1},
                                 {F_V, 2}, {F_MASS, 0}, {F_H, 0}, {F_U, 0}, {F_RHO, 0},
                                 {F_FGRADH, 0}, {F_BALS, 0}, {F_AVISC, 0}, {F_ADIFF, 0},
                                 {F_TBIN, 0}};
    for (int k = 0; k < (int)b->bundles.size(); ++k) {
        const BatchBundle &bb = b->bundles[k];
        if (bb.ncells == 0 || bb.ntargets == 0) continue;
        D64PackArgs pa{};
        pa.cells = b->d_cells + bb.cell0;
        pa.buf = (char *)dev_buf_in;
        pa.S = bb.slots;
        for (int r = 0; r < R_NUM; ++r) pa.src[r] = at(s, roles[r][0], roles[r][1]);
        pa.kernel_gamma = p->kernel_gamma;
        k_pack64<<<(unsigned)bb.ncells, 128, 0, st>>>(pa);
        if (int rc = launch_check("fp64 pack")) return rc;
        D64Args ia{};
        ia.cells = b->d_cells + bb.cell0;
        ia.targets = b->d_targets + bb.target0;
        ia.nbrs = b->d_nbrs;
        ia.in = (const char *)dev_buf_in;
        ia.S = bb.slots;
        for (int d = 0; d < 3; ++d) ia.box[d] = b->box[d];
        ia.active_bin = p->active_bin;
        const unsigned g = (unsigned)bb.ntargets;
        if (loop == SPH_DENSITY) k_count64<SPH_DENSITY><<<g, 128, 0, st>>>(ia, dev_count);
        else if (loop == SPH_GRADIENT) k_count64<SPH_GRADIENT><<<g, 128, 0, st>>>(ia, dev_count);
        else k_count64<SPH_FORCE><<<g, 128, 0, st>>>(ia, dev_count);
        if (int rc = launch_check("fp64 pair count")) return rc;
    }
    return SPH_OK;
}

// ---- neighbour-list variant of the batched cycle ---------------------------
size_t sph_batch_list_bytes(sph_batch b, int64_t chunks) {
    if (!b || chunks < 0) return 0;
    return (size_t)ListLayout::bytes((int64_t)b->items.size(), b->mask_words, chunks);
}

int sph_batch_list_build(sph_store s, sph_batch b, void *dev_buf_in, void *dev_list,
                         size_t list_bytes, const sph_params *p, void *stream) {
    if (int rc = check_store(s)) return rc;
    if (!b) return fail(SPH_EINVAL, "NULL batch handle");
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_list || !aligned256(dev_list))
        return fail(SPH_EINVAL, "buffers must be 256-byte aligned device pointers");
    const int64_t NI = (int64_t)b->items.size();
    if ((int64_t)list_bytes < ListLayout::fixed(NI, b->mask_words) + 512)
        return fail(SPH_EINVAL, "list buffer smaller than sph_batch_list_bytes(b, 0)");
    // the header is reset here too, so a plan without bundles leaves it valid
    if (int rc = cuda_check(cudaMemsetAsync(dev_list, 0, sizeof(ListHdr), (cudaStream_t)stream),
                            "reset list header"))
        return rc;
    for (int k = 0; k < (int)b->bundles.size(); ++k) {
        if (int rc = sph_batch_pack(s, b, SPH_DENSITY, k, dev_buf_in, p, stream)) return rc;
        if (int rc = sph_batch_list_build_bundle(s, b, k, dev_buf_in, dev_list, list_bytes, p,
                                                 stream))
            return rc;
    }
    return SPH_OK;
}

int sph_batch_list_count(sph_store s, sph_batch b, int bundle, const void *dev_buf_in,
                         void *dev_list, size_t list_bytes, const sph_params *p,
                         unsigned long long *dev_counts, void *stream) {
    if (int rc = check_store(s)) return rc;
    if (int rc = check_batch(b, bundle)) return rc;
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_list || !aligned256(dev_list) ||
        !dev_counts || ((uintptr_t)dev_counts & 7u))
        return fail(SPH_EINVAL, "buffers must be 256-byte aligned device pointers, the counts "
                                "8-byte aligned");
    const int64_t NI = (int64_t)b->items.size();
    if ((int64_t)list_bytes < ListLayout::fixed(NI, b->mask_words) + 512)
        return fail(SPH_EINVAL, "list buffer smaller than sph_batch_list_bytes(b, 0)");
    cudaStream_t st = (cudaStream_t)stream;
    ListView L = ListLayout::view(dev_list, NI, b->mask_words, (int64_t)list_bytes);
    if (bundle == 0)
        if (int rc = cuda_check(cudaMemsetAsync(L.hdr, 0, sizeof(ListHdr), st),
                                "reset list header"))
            return rc;
    const BatchBundle &bb = b->bundles[bundle];
    if (bb.nitems == 0) return SPH_OK;
    BInteractArgs a = interact_args(b, bundle, dev_buf_in, nullptr, p);
    if (int rc = cuda_check(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st),
                            "reset work queue"))
        return rc;
    if (b->sym && b->sym_on)
        return dispatch_blist_sym<true>(b->threads, a, L, bb.item0, dev_counts, st);
    if (b->fixed_build)
        return dispatch_blist_count_p<true>(b->threads, a, L, bb.item0, dev_counts, st);
    return dispatch_blist_count_p<false>(b->threads, a, L, bb.item0, dev_counts, st);
}

int sph_batch_list_build_bundle(sph_store s, sph_batch b, int bundle, const void *dev_buf_in,
                                void *dev_list, size_t list_bytes, const sph_params *p,
                                void *stream) {
    StageRange range_(stage_name(ST_LIST, 0));
    if (int rc = check_store(s)) return rc;
    if (int rc = check_batch(b, bundle)) return rc;
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_list || !aligned256(dev_list))
        return fail(SPH_EINVAL, "buffers must be 256-byte aligned device pointers");
    const int64_t NI = (int64_t)b->items.size();
    if ((int64_t)list_bytes < ListLayout::fixed(NI, b->mask_words) + 512)
        return fail(SPH_EINVAL, "list buffer smaller than sph_batch_list_bytes(b, 0)");
    cudaStream_t st = (cudaStream_t)stream;
    ListView L = ListLayout::view(dev_list, NI, b->mask_words, (int64_t)list_bytes);
    if (bundle == 0)
        if (int rc = cuda_check(cudaMemsetAsync(L.hdr, 0, sizeof(ListHdr), st),
                                "reset list header"))
            return rc;
    const BatchBundle &bb = b->bundles[bundle];
    if (bb.nitems == 0) return SPH_OK;
    BInteractArgs a = interact_args(b, bundle, dev_buf_in, nullptr, p);
    if (int rc = cuda_check(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st),
                            "reset work queue"))
        return rc;
    return dispatch_blist(b, a, L, bb.item0, st);
}

int sph_batch_list_status(const void *dev_list, int64_t *chunks_needed, int *overflow) {
    if (!dev_list || !chunks_needed || !overflow) return fail(SPH_EINVAL, "NULL argument");
    ListHdr h{};
    if (int rc = cuda_check(cudaMemcpy(&h, dev_list, sizeof(h), cudaMemcpyDeviceToHost),
                            "read list header"))
        return rc;
    *chunks_needed = (int64_t)h.chunks_used;
    *overflow = (int)h.overflow;
    return SPH_OK;
}

size_t sph_batch_x64_bytes(sph_batch b) {
    if (!b) return 0;
    return 3 * (size_t)((8 * b->max_slots + 255) / 256 * 256);
}

int sph_batch_offload_step_list_x64(sph_store s, sph_batch b, void *dev_buf_in,
                                    void *dev_buf_out, void *dev_list, size_t list_bytes,
                                    void *dev_x64, size_t x64_bytes, const sph_params *p,
                                    void *stream) {
    if (int rc = check_store(s)) return rc;
    if (!b) return fail(SPH_EINVAL, "NULL batch handle");
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_buf_out || !aligned256(dev_buf_out) ||
        !dev_list || !aligned256(dev_list) || !dev_x64 || !aligned256(dev_x64))
        return fail(SPH_EINVAL, "buffers must be 256-byte aligned device pointers");
    if (x64_bytes < sph_batch_x64_bytes(b))
        return fail(SPH_EINVAL, "FP64 position buffer holds %zu bytes, needs %zu", x64_bytes,
                    sph_batch_x64_bytes(b));
    const int64_t NI = (int64_t)b->items.size();
    if ((int64_t)list_bytes < ListLayout::fixed(NI, b->mask_words) + 512)
        return fail(SPH_EINVAL, "list buffer smaller than sph_batch_list_bytes(b, 0)");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(cudaMemsetAsync(dev_list, 0, sizeof(ListHdr), st),
                            "reset list header"))
        return rc;
    const size_t lane = (size_t)((8 * b->max_slots + 255) / 256 * 256);
    double *xd[3] = {(double *)dev_x64, (double *)((char *)dev_x64 + lane),
                     (double *)((char *)dev_x64 + 2 * lane)};
    const CompPtr x0 = at(s, F_X, 0), x1 = at(s, F_X, 1), x2 = at(s, F_X, 2);
    ListView L = ListLayout::view(dev_list, NI, b->mask_words, (int64_t)list_bytes);
    for (int loop = 0; loop < 3; ++loop)
        for (int k = 0; k < (int)b->bundles.size(); ++k) {
            const BatchBundle &bb = b->bundles[k];
            if (int rc = sph_batch_pack_list(s, b, loop, k, dev_buf_in, p, stream)) return rc;
            if (bb.slots > 0) {
                const int64_t S = bb.slots;
                const int64_t perm_off = loop == SPH_DENSITY ? BLayout<SPH_DENSITY>::perm(S)
                                         : loop == SPH_GRADIENT ? BLayout<SPH_GRADIENT>::perm(S)
                                                                : BLayout<SPH_FORCE>::perm(S);
                k_pack_x64<<<grid_for(S, 256), 256, 0, st>>>(
                    (const int32_t *)((const char *)dev_buf_in + perm_off), S, x0, x1, x2, xd[0],
                    xd[1], xd[2]);
                if (int rc = launch_check("FP64 positions")) return rc;
            }
            if (loop == SPH_DENSITY)
                if (int rc = sph_batch_list_build_bundle(s, b, k, dev_buf_in, dev_list,
                                                         list_bytes, p, stream))
                    return rc;
            if (bb.nitems > 0) {
                BInteractArgs a = interact_args(b, k, dev_buf_in, dev_buf_out, p);
                for (int d = 0; d < 3; ++d) {
                    a.xd[d] = xd[d];
                    a.box_d[d] = b->box[d];
                    a.half_d[d] = 0.5 * b->box[d];
                }
                if (int rc = cuda_check(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st),
                                        "reset work queue"))
                    return rc;
                int rc = loop == SPH_DENSITY    ? dispatch_bloop64<SPH_DENSITY>(b, a, L, bb.item0, st)
                         : loop == SPH_GRADIENT ? dispatch_bloop64<SPH_GRADIENT>(b, a, L, bb.item0, st)
                                                : dispatch_bloop64<SPH_FORCE>(b, a, L, bb.item0, st);
                if (rc) return rc;
            }
            if (int rc = sph_batch_unpack_write(s, b, loop, k, dev_buf_out, dev_buf_in, p,
                                                loop == SPH_DENSITY ? 1 : 0, stream))
                return rc;
        }
    return SPH_OK;
}

int sph_batch_list_interact(sph_batch b, int loop, int bundle, const void *dev_buf_in,
                            void *dev_buf_out, const void *dev_list, size_t list_bytes,
                            const sph_params *p, void *stream) {
    StageRange range_(stage_name(ST_INTERACT, loop));
    if (int rc = check_batch(b, bundle)) return rc;
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_buf_out || !aligned256(dev_buf_out) ||
        !dev_list || !aligned256(dev_list))
        return fail(SPH_EINVAL, "buffers must be 256-byte aligned device pointers");
    const int64_t NI = (int64_t)b->items.size();
    if ((int64_t)list_bytes < ListLayout::fixed(NI, b->mask_words) + 512)
        return fail(SPH_EINVAL, "list buffer smaller than sph_batch_list_bytes(b, 0)");
    const BatchBundle &bb = b->bundles[bundle];
    if (bb.nitems == 0) return SPH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    ListView L = ListLayout::view(const_cast<void *>(dev_list), NI, b->mask_words, (int64_t)list_bytes);
    BInteractArgs a = interact_args(b, bundle, dev_buf_in, dev_buf_out, p);
    if (int rc = cuda_check(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st),
                            "reset work queue"))
        return rc;
    if (loop == SPH_DENSITY) return dispatch_bloop<SPH_DENSITY>(b, a, L, bb.item0, st);
    if (loop == SPH_GRADIENT) return dispatch_bloop<SPH_GRADIENT>(b, a, L, bb.item0, st);
    return dispatch_bloop<SPH_FORCE>(b, a, L, bb.item0, st);
}

int sph_batch_offload_loop_list(sph_store s, sph_batch b, int loop, void *dev_buf_in,
                                void *dev_buf_out, const void *dev_list, size_t list_bytes,
                                const sph_params *p, void *stream) {
    if (int rc = check_store(s)) return rc;
    if (!b) return fail(SPH_EINVAL, "NULL batch handle");
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_buf_out || !aligned256(dev_buf_out) ||
        !dev_list || !aligned256(dev_list))
        return fail(SPH_EINVAL, "buffers must be 256-byte aligned device pointers");
    if ((int64_t)list_bytes < ListLayout::fixed((int64_t)b->items.size(), b->mask_words) + 512)
        return fail(SPH_EINVAL, "list buffer smaller than sph_batch_list_bytes(b, 0)");
    for (int k = 0; k < (int)b->bundles.size(); ++k) {
        if (int rc = sph_batch_pack_list(s, b, loop, k, dev_buf_in, p, stream)) return rc;
        if (int rc = sph_batch_list_interact(b, loop, k, dev_buf_in, dev_buf_out, dev_list,
                                             list_bytes, p, stream))
            return rc;
        if (int rc = sph_batch_unpack_write(s, b, loop, k, dev_buf_out, dev_buf_in, p, 1,
                                            stream))
            return rc;
    }
    return SPH_OK;
}

int sph_batch_offload_step_list(sph_store s, sph_batch b, void *dev_buf_in, void *dev_buf_out,
                                void *dev_list, size_t list_bytes, const sph_params *p,
                                void *stream) {
    if (int rc = check_store(s)) return rc;
    if (!b) return fail(SPH_EINVAL, "NULL batch handle");
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_buf_out || !aligned256(dev_buf_out) ||
        !dev_list || !aligned256(dev_list))
        return fail(SPH_EINVAL, "buffers must be 256-byte aligned device pointers");
    if ((int64_t)list_bytes < ListLayout::fixed((int64_t)b->items.size(), b->mask_words) + 512)
        return fail(SPH_EINVAL, "list buffer smaller than sph_batch_list_bytes(b, 0)");
    if (int rc = cuda_check(cudaMemsetAsync(dev_list, 0, sizeof(ListHdr), (cudaStream_t)stream),
                            "reset list header"))
        return rc;
    for (int k = 0; k < (int)b->bundles.size(); ++k) {
        if (int rc = sph_batch_pack_list(s, b, SPH_DENSITY, k, dev_buf_in, p, stream)) return rc;
        if (int rc = sph_batch_list_build_bundle(s, b, k, dev_buf_in, dev_list, list_bytes, p,
                                                 stream))
            return rc;
        if (int rc = sph_batch_list_interact(b, SPH_DENSITY, k, dev_buf_in, dev_buf_out,
                                             dev_list, list_bytes, p, stream))
            return rc;
        if (int rc = sph_batch_unpack_write(s, b, SPH_DENSITY, k, dev_buf_out, dev_buf_in, p, 1,
                                            stream))
            return rc;
    }
    for (int loop : {SPH_GRADIENT, SPH_FORCE})
        if (int rc = sph_batch_offload_loop_list(s, b, loop, dev_buf_in, dev_buf_out, dev_list,
                                                 list_bytes, p, stream))
            return rc;
    return SPH_OK;
}


// ---- adjoint of density -> ghost -> force ----------------------------------
size_t sph_batch_adjoint_bytes(sph_batch b) {
    if (!b || b->bundles.size() != 1) return 0;
    const int64_t S = b->bundles[0].slots;
    return (size_t)(((S * 16 * (kAdjRec + 4)) + 255) / 256 * 256 + 256);
}

int sph_batch_adjoint(sph_store s, sph_batch b, void *dev_buf_in, const void *dev_list,
                      size_t list_bytes, void *dev_scratch, size_t scratch_bytes,
                      const int64_t *dev_store_perm, const float *dev_abar,
                      const float *dev_ebar, double *dev_gx, float *dev_gm, float *dev_gu,
                      const sph_params *p, void *stream) {
    StageRange range_(stage_name(ST_ADJOINT, 0));
    if (int rc = check_store(s)) return rc;
    if (!b) return fail(SPH_EINVAL, "NULL batch handle");
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (b->bundles.size() != 1)
        return fail(SPH_EUNSUPPORTED, "the adjoint needs a plan of one bundle "
                                      "(max_target_cells <= 0)");
    if (!dev_buf_in || !aligned256(dev_buf_in) || !dev_list || !aligned256(dev_list) ||
        !dev_scratch || !aligned256(dev_scratch))
        return fail(SPH_EINVAL, "buffers must be 256-byte aligned device pointers");
    if (!dev_abar || !dev_ebar || !dev_gx || !dev_gm || !dev_gu)
        return fail(SPH_EINVAL, "NULL adjoint array");
    if (scratch_bytes < sph_batch_adjoint_bytes(b))
        return fail(SPH_EINVAL, "scratch smaller than sph_batch_adjoint_bytes");
    const int64_t NI = (int64_t)b->items.size();
    if ((int64_t)list_bytes < ListLayout::fixed(NI, b->mask_words) + 512)
        return fail(SPH_EINVAL, "list buffer smaller than sph_batch_list_bytes(b, 0)");
    const BatchBundle &bb = b->bundles[0];
    if (bb.nitems == 0) return SPH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // the slot order of the lists: the bundle's density pack
    if (int rc = sph_batch_pack(s, b, SPH_DENSITY, 0, dev_buf_in, p, stream)) return rc;
    AdjArgs a{};
    a.cells = b->d_cells + bb.cell0;
    a.targets = b->d_targets + bb.target0;
    a.items = b->d_items + bb.item0;
    a.counter = b->d_counter;
    a.nitems = (int)bb.nitems;
    a.item0 = bb.item0;
    a.L = ListLayout::view(const_cast<void *>(dev_list), NI, b->mask_words, (int64_t)list_bytes);
    a.S = bb.slots;
    a.perm = reinterpret_cast<const int32_t *>((const char *)dev_buf_in +
                                               BLayout<SPH_DENSITY>::perm(bb.slots));
    a.store_perm = dev_store_perm;
    char *sc = (char *)dev_scratch;
    a.rec = reinterpret_cast<float4 *>(sc);
    a.g = a.rec + kAdjRec * bb.slots;
    a.sg = a.g + 2 * bb.slots;
    const int roles[A_NUM][2] = {{F_X, 0}, {F_X, 1}, {F_X, 2}, {F_V, 0}, {F_V, 1}, {F_V, 2},
                                 {F_MASS, 0}, {F_H, 0}, {F_U, 0}, {F_RHO, 0}, {F_FGRADH, 0},
                                 {F_BALS, 0}, {F_AVISC, 0}, {F_ADIFF, 0}, {F_CS, 0},
                                 {F_PRES, 0}, {F_TBIN, 0}, {F_RHODH, 0}, {F_DIVV, 0},
                                 {F_ROTV, 0}, {F_ROTV, 1}, {F_ROTV, 2}, {F_WCOUNT, 0}};
    for (int r = 0; r < A_NUM; ++r) a.f[r] = at(s, roles[r][0], roles[r][1]);
    a.abar = dev_abar;
    a.ebar = dev_ebar;
    a.gx_out = dev_gx;
    a.gm_out = dev_gm;
    a.gu_out = dev_gu;
    a.kernel_gamma = (float)p->kernel_gamma;
    a.gamma = (float)p->gamma;
    a.beta = (float)p->beta_visc;
    a.eps = (float)p->balsara_eps;
    for (int d = 0; d < 3; ++d) {
        a.shift_hi[d] = (float)b->box[d];
        a.shift_lo[d] = (float)(b->box[d] - (double)a.shift_hi[d]);
        a.half[d] = (float)(0.5 * b->box[d]);
    }
    a.active_bin = p->active_bin;
    const unsigned g = grid_for(bb.slots, 256);
    k_adj_pack<<<g, 256, 0, st>>>(a);
    if (int rc = launch_check("adjoint pack")) return rc;
    if (int rc = cuda_check(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st), "queue"))
        return rc;
    if (int rc = launch_persistent(k_adj_pairs<0>, 128, a.nitems, st, "force adjoint", a))
        return rc;
    k_adj_ghost<<<g, 256, 0, st>>>(a);
    if (int rc = launch_check("ghost adjoint")) return rc;
    if (int rc = cuda_check(cudaMemsetAsync(a.counter, 0, sizeof(unsigned int), st), "queue"))
        return rc;
    if (int rc = launch_persistent(k_adj_pairs<1>, 128, a.nitems, st, "density adjoint", a))
        return rc;
    k_adj_scatter<<<g, 256, 0, st>>>(a);
    return launch_check("adjoint scatter");
}

// ---- host-staged batched cycle ----------------------------------------------
int sph_batch_offload_loop_host(sph_store s, sph_batch b, int loop, void *const host_in[2],
                                void *const host_out[2], void *const dev_in[2],
                                void *const dev_out[2], const sph_params *p,
                                void *const streams[2], int nthreads) {
    if (int rc = check_host_store(s)) return rc;
    if (!b) return fail(SPH_EINVAL, "NULL batch handle");
    if (int rc = check_loop(loop)) return rc;
    if (int rc = check_params(p)) return rc;
    if (s->n != b->n) return fail(SPH_EINVAL, "store and batch disagree on particle count");
    if (!host_in || !host_out || !dev_in || !dev_out || !streams)
        return fail(SPH_EINVAL, "NULL buffer or stream array");
    for (int k = 0; k < 2; ++k)
        if (!aligned256(host_in[k]) || !aligned256(host_out[k]) || !aligned256(dev_in[k]) ||
            !aligned256(dev_out[k]) || !host_in[k] || !host_out[k] || !dev_in[k] || !dev_out[k])
            return fail(SPH_EINVAL, "buffers must be non-NULL and 256-byte aligned");
    if (int rc = host_init(s, loop, p->active_bin, nthreads)) return rc;
    const int nb = (int)b->bundles.size();
    cudaStream_t st[2] = {(cudaStream_t)streams[0], (cudaStream_t)streams[1]};
    cudaEvent_t done[2] = {nullptr, nullptr};
    int rc = SPH_OK;
    for (int k = 0; k < 2 && rc == SPH_OK; ++k)
        rc = cuda_check(cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming), "event");
    std::vector<int> ids;
    for (int bi = 0; bi < nb; ++bi)
        if (b->bundles[bi].nitems > 0) ids.push_back(bi);
    const int nq = (int)ids.size();
    for (int q = 0; q < nq && rc == SPH_OK; ++q) {
        const int k = q & 1, bi = ids[q];
        // buffers k were last used by bundle q-2, whose results were folded
        // after its event completed in the previous iteration
        if ((rc = host_batch_pack(s, b, loop, bi, (char *)host_in[k], p, nthreads))) break;
        const size_t in_b = (size_t)host_batch_in_bytes(b, loop, bi);
        const size_t out_b = (size_t)host_batch_out_bytes(b, loop, bi);
        if ((rc = cuda_check(cudaMemcpyAsync(dev_in[k], host_in[k], in_b,
                                             cudaMemcpyHostToDevice, st[k]), "H2D")))
            break;
        if ((rc = sph_batch_interact(b, loop, bi, dev_in[k], dev_out[k], p, st[k]))) break;
        if ((rc = cuda_check(cudaMemcpyAsync(host_out[k], dev_out[k], out_b,
                                             cudaMemcpyDeviceToHost, st[k]), "D2H")))
            break;
        if ((rc = cuda_check(cudaEventRecord(done[k], st[k]), "event record"))) break;
        if (q >= 1) {
            if ((rc = cuda_check(cudaEventSynchronize(done[k ^ 1]), "event wait"))) break;
            if ((rc = host_batch_unpack(s, b, loop, ids[q - 1], (const char *)host_out[k ^ 1],
                                        nthreads)))
                break;
        }
    }
    if (rc == SPH_OK && nq > 0) {
        const int k = (nq - 1) & 1;
        rc = cuda_check(cudaEventSynchronize(done[k]), "event wait");
        if (rc == SPH_OK)
            rc = host_batch_unpack(s, b, loop, ids[nq - 1], (const char *)host_out[k], nthreads);
    }
    if (rc != SPH_OK) {
        cudaStreamSynchronize(st[0]);
        cudaStreamSynchronize(st[1]);
    }
    for (int k = 0; k < 2; ++k)
        if (done[k]) cudaEventDestroy(done[k]);
    if (rc == SPH_OK && loop == SPH_DENSITY) rc = sph_ghost_host(s, SPH_DENSITY, p, nthreads);
    return rc;
}

int sph_fault_inject(int site, int countdown) {
    if (site < 0 || site > SPH_FAULT_COPY || countdown < 0)
        return fail(SPH_EINVAL, "fault_inject: unknown site or negative countdown");
    g_fault_countdown.store(countdown);
    g_fault_site.store(countdown > 0 ? site : 0);
    return SPH_OK;
}
}  // extern "C"
