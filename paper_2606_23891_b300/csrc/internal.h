// Internal declarations of libsph: layout engine, task builder, device
// records.  Not part of the public C-ABI (include/sph.h).
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "sph.h"

namespace sph {

// Logical fields, in the order of the sph_fields struct; F_BALLAST stands for
// the struct members no loop touches.
enum FieldId {
    F_X = 0, F_V, F_A, F_MASS, F_H, F_U, F_UDT, F_RHO, F_TBIN, F_AVISC,
    F_ADIFF, F_RHODH, F_WCOUNT, F_WCOUNTDH, F_DIVV, F_ROTV, F_FGRADH, F_PRES,
    F_CS, F_BALS, F_VSIGG, F_LAPU, F_HDT, F_VSIG, F_ID, F_BALLAST, F_NUM
};

enum TypeClass { T_DOUBLE = 0, T_FLOAT = 1, T_INT = 2 };

struct FieldInfo {
    int elem;   // bytes per component
    int count;  // components
    int cls;    // TypeClass
};
extern const FieldInfo kFields[F_NUM];

struct Member {
    int field;
    int comp;    // -1: the whole field; >= 0: a single component (SoA)
    int offset;  // byte offset inside the record
};

struct Group {
    std::vector<Member> mem;
    int record = 0;     // record bytes
    int64_t base = 0;   // byte offset of the group's array inside the store
};

struct Layout {
    int id = -1;
    uint64_t seed = 0;
    std::vector<Group> groups;
    int view_group[3] = {-1, -1, -1};  // group each loop's pack reads first
};

// Layout engine (layout.cpp).
int build_layout(int layout, uint64_t seed, int64_t n, Layout *out);
int64_t layout_bytes(const Layout &L, int64_t n);

// Element address of (field, comp) of particle p: ptr + p * stride.
struct CompPtr {
    char *ptr;
    long long stride;
};
bool locate(const Layout &L, char *mem, int field, int comp, CompPtr *out);
// Every copy of (field, comp) (replicated layouts hold some inputs twice);
// returns the number found (at most max).
int locate_all(const Layout &L, char *mem, int field, int comp, CompPtr *out, int max);
// The copy a loop's pack reads: the one in the loop's view group when the
// layout names one and it holds the field, else the first.
bool locate_view(const Layout &L, char *mem, int field, int comp, int loop, CompPtr *out);

// Error reporting (api.cu).
int fail(int status, const char *fmt, ...);

}  // namespace sph

// One task as the kernels see it (24 bytes).  pi/ni: first particle (store
// index) and count of cell ci; pj/nj the same for cj (nj = 0: self task).
// slot: first slot of the task inside its bundle.  shift: periodic shift of
// cj, per dimension (code + 1) in 2-bit fields (x: bits 0-1, y: 2-3, z: 4-5);
// bits 6-11 hold the cell offset d from ci to cj the same way (0 for self).
struct TaskDev {
    int32_t pi, ni, pj, nj, slot, shift;
};

// One cell of a bundle as the unpack kernel sees it: particles [p0, p0+n),
// and ne entries at e0 (relative to the bundle's entry base), each the slot
// of the cell's first particle in one task, in increasing task order.
struct UCellDev {
    int32_t p0, n, e0, ne;
};

struct sph_store_s {
    int64_t n = 0;
    sph::Layout layout;
    char *mem = nullptr;
    size_t bytes = 0;
    bool host = false;  // store in host memory (host-staged path)
};

struct sph_tasks_s {
    int64_t n = 0;
    int32_t ncell[3] = {0, 0, 0};
    double box[3] = {0, 0, 0};
    std::vector<int64_t> cell_start;    // ncells + 1
    std::vector<int32_t> ci, cj;        // per task
    std::vector<int8_t> shift;          // 3 per task
    std::vector<int64_t> bundle_start;  // nbundles + 1
    std::vector<int64_t> bundle_slots;  // per bundle
    std::vector<TaskDev> tdev;          // per task (slot is bundle-relative)
    std::vector<int64_t> ucell_begin;   // nbundles + 1, into ucells
    std::vector<int64_t> entry_begin;   // nbundles + 1, into entries
    std::vector<UCellDev> ucells;
    std::vector<int32_t> entries;
    int64_t max_cell = 0;
    // device copies (sph_tasks_upload)
    TaskDev *d_tasks = nullptr;
    UCellDev *d_ucells = nullptr;
    int32_t *d_entries = nullptr;
    int device = -1;
};

// ---- batched (cell-dedup) pipeline records --------------------------------
// A cell of a batched bundle: particles [p0, p0+n) of the store, packed at
// bundle slots [slot, slot+n) (octant-sorted inside the cell).  hlim: the
// largest support H the plan holds for the cell's particles (grid: the cell
// edge; tree: the leaf's largest support when the plan was built); the
// density pack reports a larger one (the plan must then be rebuilt).
struct BCellDev {
    int32_t p0, n, slot;
    float hlim;
};
// A target cell: its local cell index and its neighbour entries
// [nb0, nb0 + nnb) of the plan's neighbour list.
struct BTargetDev {
    int32_t cell, nb0, nnb, pad;
};
// A neighbour entry: a local cell whose particles may interact with the
// target's, and the periodic shift of those particles (code + 1 per
// dimension in 2-bit fields).  A cell may appear with several shifts.
struct BNbrDev {
    int32_t cell, code;
};
// A work item (one warp): particles [i0, i0 + 32) of target `target`.
struct BItemDev {
    int32_t target, i0;
};
// A backward neighbour of a target in the symmetric list build: where the
// masks of the (neighbour, target) pair start (the target's first chunk
// word), the stride between the neighbour's 32-particle chunks, and the
// neighbour's first slot and particle count.
struct RevEntDev {
    long long mrow;
    int32_t stride, slot, n, pad;
};
struct BatchBundle {
    int64_t cell0 = 0, ncells = 0, slots = 0;
    int64_t target0 = 0, ntargets = 0;
    int64_t item0 = 0, nitems = 0;
};

struct sph_batch_s {
    int64_t n = 0;
    int threads = 128;
    double box[3] = {0, 0, 0};
    std::vector<BatchBundle> bundles;
    std::vector<BCellDev> cells;
    std::vector<BTargetDev> targets;
    std::vector<BItemDev> items;
    std::vector<BNbrDev> nbrs;
    int64_t max_slots = 0, max_targets = 0;
    int kind = 0;                 // 0: uniform cell grid, 1: adaptive octree leaves
    // the list build may use fixed-point separations: every cell or leaf
    // extent plus the largest support stays below half the box
    bool fixed_build = false;
    int64_t plan_cells = 0, plan_max_cell = 0, plan_nbrs = 0;
    // symmetric list build (one bundle, fixed-point path, every cell pair in
    // both targets' entries): each cell pair is tested once, from the lower
    // cell ("forward" entries), whose warps store their hit masks; the higher
    // cell's lists get the pair by transposing them.  naux: per entry, the
    // forward ordinal (forward entries) or the ordinal of this target among
    // the other cell's forward entries (backward ones), -1 for self; mbase:
    // per target, its first mask word; targets' pad field: forward entries.
    bool sym = false;
    bool sym_on = true;                 // sph_batch_list_symmetric
    int sym_words = 0;                  // mask words per entry and chunk (32 candidates each)
    int64_t mask_words = 0;             // mask region of the list buffer (0 when off)
    std::vector<int32_t> naux;
    std::vector<int64_t> mbase;
    std::vector<RevEntDev> rev;         // per target, its backward neighbours in entry order
    std::vector<int32_t> rev_start;     // per target (+1): its first entry of rev
    int32_t *d_naux = nullptr;
    long long *d_mbase = nullptr;
    RevEntDev *d_rev = nullptr;
    int32_t *d_rev_start = nullptr;
    BCellDev *d_cells = nullptr;
    BTargetDev *d_targets = nullptr;
    BNbrDev *d_nbrs = nullptr;
    BItemDev *d_items = nullptr;
    unsigned int *d_counter = nullptr;  // work-queue head, one per bundle
};

namespace sph {
int build_batch(const sph_tasks_s *T, const sph_batch_params *bp, sph_batch_s *B);
// The symmetric list build's plan data (sym, naux, mbase, mask_words).
void build_sym(sph_batch_s *B);
int build_batch_tree(int64_t n, const double *x, const float *h, const sph_tree_params *tp,
                     const sph_batch_params *bp, int64_t *perm_out, sph_batch_s *B);
int tree_plan_host(int64_t n, const double *x, const float *h, const sph_tree_params *tp,
                   int64_t *perm_out, int64_t *leaf_start, int64_t *nleaf_out,
                   int64_t *nb_start, int32_t *nb, int64_t nb_cap, int64_t *nnb_out);

int build_tasks(int64_t n, const double *x, const float *h,
                const sph_grid_params *gp, int64_t *perm_out, sph_tasks_s *T);

// Host-staged path (host_path.cpp): OpenMP over tasks / cells / particles.
int host_pack(sph_store s, sph_tasks t, int loop, int b, char *buf, int nthreads);
int host_unpack(sph_store s, sph_tasks t, int loop, int b, const char *buf, int nthreads);
int host_init(sph_store s, int loop, int active_bin, int nthreads);
int host_pack_fission(sph_store s, sph_tasks t, int loop, int b, char *buf, int fission,
                      int nthreads);
int host_unpack_fission(sph_store s, sph_tasks t, int loop, int b, const char *buf, int fission,
                        int nthreads);
int host_ghost(sph_store s, float kernel_gamma, float gamma, float balsara_eps, int nthreads);
int host_copy_fields(sph_store s, const sph_fields *f, const int64_t *perm, int to_store,
                     int nthreads);

// Packed-buffer lanes of Sec. 2.3 buffers: sizes of each lane of `loop`
// (in_or_out 0 = pack buffer, 1 = result buffer); returns the lane count.
int lane_sizes(int loop, int in_or_out, int64_t *sizes);
// Byte offsets of the lanes for S slots; returns the total bytes.
int64_t lane_offsets(int loop, int in_or_out, int64_t S, int64_t *offsets);
}  // namespace sph
