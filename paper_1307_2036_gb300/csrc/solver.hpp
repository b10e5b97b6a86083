// Internal host-side types of the ellsolve driver.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "common.cuh"
#include "ellsolve.h"

namespace ells {

struct Error : std::runtime_error {
    ellsolve_status status;
    Error(ellsolve_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

void check_cuda(cudaError_t e, const char *what);
void set_last_error(const std::string &m);

// Owning device allocation.
// A device allocation.  alloc() keeps the current block when it is large
// enough (bytes is the size asked for, cap the size allocated), so that plans
// rebuilt for a changed batch do not free and allocate again.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0, cap = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), cap(o.cap) {
        o.p = nullptr;
        o.bytes = o.cap = 0;
    }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            reset();
            p = o.p;
            bytes = o.bytes;
            cap = o.cap;
            o.p = nullptr;
            o.bytes = o.cap = 0;
        }
        return *this;
    }
    ~DevBuf() { reset(); }
    void alloc(size_t b);
    void reset();
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

// Device geometry of one level: column metrics and connectivity (FP64 and FP32).
struct LevelGeom {
    int n = 0, ncol = 0;
    double area_sq = 0.0;  // sum of the squared cell areas
    DevBuf area64, tr64, area32, tr32, nbr, pst;
};

// The hierarchy of one grid; shared by every problem on that grid and kept
// resident while any of them lives (process-wide cache keyed by the grid).
struct Geometry {
    int kind = 0, P = 1, mapping = 0;
    std::vector<LevelGeom> lev;
    size_t bytes = 0;
};
std::shared_ptr<const Geometry> geometry_for(const ellsolve_grid &g, int coarsest_min,
                                             int max_levels, cudaStream_t s);

// Launch shape of one level's kernels.  No result depends on it: the same
// arithmetic runs in another schedule.
struct LevelShape {
    int ctas = 3;   // twisted smoother: resident CTAs per SM cap (0: as many as fit)
    int ring = 8;   // twisted smoother: staging ring depth, 4 or 8 steps
    int tmem = 0;   // twisted smoother: f' in tensor memory 0 on launches of >= 152
                    // CTAs, 1 always (n_z <= 256), 2 never
    int staged = 0;  // fully staged smoother: 0 on launches of fewer than 152 blocks
                     // of 128 columns, 1 always, 2 never (where it fits)
    int restrict_chunk = 608;  // residual + restriction from this level, and the
    int prolong_chunk = 608;   // prolongation onto it: launches of fewer blocks are split
                               // along the vertical until about this many exist
};

// Device vectors of one multigrid level of one problem.
struct LevelStore {
    int n = 0, ncol = 0;
    const LevelGeom *geo = nullptr;
    DevBuf u64[2], b64, aux64;
    DevBuf u32[2], b32, aux32;
};

// Device bytes a problem needs beyond its (shared) geometry.
size_t problem_vector_bytes(const ellsolve_grid &g, const ellsolve_opts &o);
size_t geometry_bytes(const ellsolve_grid &g, const ellsolve_opts &o);

// One launch of a V-cycle program.
struct Op {
    enum Kind { kSmooth, kRestrict, kRestrictRhs, kProlong, kMemset } kind = kSmooth;
    int off = 0, n = 0;       // range in the plan's item array
    double rho = 1.0;         // smoother damping
    int max_nz = 0;           // largest nz among the items
    bool finest = false;      // smooths a finest level (profiled)
    double bytes = 0.0;       // algorithmic bytes of the finest-level work
    int zero_mode = 0;        // smoother items: 0 none / 1 all start from zero, 2 mixed
    bool rows_ok = false;     // every level in the op suits the row-staged FP32 smoother
    bool aligned = false;     // every level in the op has n % 32 == 0
    bool part = false;        // every level in the op takes the partitioned line solve
    int tune = 0;             // level whose launch shape the op takes (its first item's)
    int member = 0, level = 0, buf = 0;  // kMemset target
};

struct Program {
    std::vector<Op> ops;
    std::vector<int> fine_cur_out;  // finest-level buffer per member after the cycle
    int update_off = 0, update_n = 0;
};

struct Problem;

// The launch program of a set of problems ("members") solved together: every
// kernel of the V-cycle is one launch over the items of all members.
struct Plan {
    Plan() = default;
    Plan(const Plan &) = delete;
    Plan &operator=(const Plan &) = delete;
    std::vector<Problem *> mem;
    int precision = 1;
    std::vector<int> base;  // first descriptor of each member
    int maxlev = 0, maxnz = 0;
    DevBuf desc64, desc32;  // level descriptors, member-major
    DevBuf outer64, fine32; // finest-level descriptors per member for the refinement
    std::vector<Lv<double>> stage64;
    std::vector<Lv<float>> stage32;
    std::vector<double> stage_scales;
    std::vector<Item> items;
    DevBuf ditems;
    bool items_dirty = true;
    std::map<std::string, Program> programs;
    int outer_off = 0, outer_n = 0;   // finest columns, lv = member
    int norm_off[2] = {0, 0}, norm_n = 0;  // finest columns, lv = descriptor, u[0] / u[1]
    std::vector<int> outer_first;     // per-member ranges of outer items
    DevBuf dfirst, partials, partials2, partials3, norms, scales, counts, active;
    std::vector<int> stage_active;
    std::vector<double> host_norms;       // [3 M]: norms, magnitudes, update norms
    double *hnorms = nullptr;             // mapped pinned staging of the device norms [4 M]
    double *hnorms_dev = nullptr;         // its device address
    size_t hnorms_n = 0;
    cudaGraphExec_t gexec = nullptr;
    int graph_launches = 0;

    ~Plan();
    void build(const std::vector<Problem *> &members, int prec);
    const Program &program(bool fine_zero, const std::vector<int> &fine_cur);
    void sync_items();
    void drop_graph();
};

struct Problem {
    ellsolve_grid grid{};
    ellsolve_opts opts{};
    double omega2 = 0, lambda2 = 0;
    std::vector<double> r;
    int nz = 0, P = 1, nlev = 0;
    size_t N = 0;
    // ||A_P V_k||_2 over the finest unknowns: the norm of the right-hand side
    // b = A_P V_k f for f = 1 (its magnitude fixes a first refinement scale)
    double b_unit_norm = 0.0;
    cudaStream_t stream = nullptr;      // the caller's stream: all work is ordered on it
    int device = 0;                     // the device current at creation (owns every buffer)
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
    std::shared_ptr<const Geometry> geom;
    std::vector<LevelStore> lev;
    DevBuf V64, g64, V32, g32;
    std::vector<Lv<double>> h64;
    std::vector<Lv<float>> h32;
    int fine_cur = 0;
    DevBuf cg[4], cg_scal;
    std::unique_ptr<Plan> plan, batch_plan;
    uint64_t launches = 0;
    bool capturing = false;
    // CUDA-event timing of the finest-level smoother launches
    bool prof = false;
    std::vector<cudaEvent_t> ev_free, ev_graph;
    int ev_next = 0, ev_graph_used = 0;
    std::vector<LevelShape> shape;  // launch shape per level (set by the autotuner)
    const LevelShape &level_shape(int level) const {
        return shape[size_t(level < nlev ? level : nlev - 1)];
    }
    double prof_ms = 0.0, prof_bytes = 0.0;
    long prof_count = 0;
    std::vector<double> ev_free_bytes, ev_graph_bytes;  // bytes per recorded pair

    ~Problem();
    void build(const ellsolve_grid &g, double w2, double l2, const double *r_levels,
               const ellsolve_opts &o, cudaStream_t s, const double *p_cell = nullptr,
               const double *q_face = nullptr);
    // new omega^2, lambda^2, radial levels and (nullable) vertical profiles on
    // the same grid and nz (reuse)
    void rebind(double w2, double l2, const double *r_levels, const double *p_cell = nullptr,
                const double *q_face = nullptr);
    std::vector<double> p_cell, q_face;  // vertical background profiles (empty: none)
    Plan &single_plan();
    size_t footprint_bytes() const;
    void prof_mark_begin(cudaStream_t s);
    void prof_mark_end(cudaStream_t s, double bytes);
    void prof_collect(bool graph_replayed);
};

// Per-member state of an iterative-refinement solve.
struct MemberRun {
    const double *f = nullptr;  // pointwise right-hand side (device)
    double *x = nullptr;        // solution (device)
    double rtol = 0.0;
    int maxit = 0;
    double bnorm = 0.0, rel = 1.0;
    int iters = 0;
    std::vector<double> hist;
    bool active = true;
    double scale_cur = 1.0, scale_next = 1.0;
    // refinement residual: 1 tracked (double-float update), 2 recomputed in
    // FP64; errb bounds |tracked - true residual| (2-norm), magx ~ || |A| |x| ||
    int mode = 1;
    double errb = 0.0, magx = 0.0;
    // norms of the first, the one but last and the latest update of x (error estimate)
    double dx_first = 0.0, dx_prev = 0.0, dx_last = 0.0;
    // x = 0 and not yet written: the first tracked update writes e / s without
    // reading x (so x is not cleared beforehand); ir_zero_unwritten clears it
    // for a member that stops before any update
    bool x_zero = false;
};

void ir_bind(Plan &pl, const std::vector<MemberRun *> &run);
void ir_start(Plan &pl, std::vector<MemberRun *> &run, int m0, int m1, bool keep_x);
void ir_advance(Plan &pl, std::vector<MemberRun *> &run, bool use_graph);
// writes x = 0 (on the plan's stream) for the finished members whose x was
// never written (no update ran); true when it enqueued any
bool ir_zero_unwritten(Plan &pl, const std::vector<MemberRun *> &run);
ellsolve_status run_result(const MemberRun &r, double secs, ellsolve_result *res);

// One line-smoother launch: the twisted FP32 kernel where `rows_ok`, else the
// generic kernel; `level`: whose launch shape to take.  The items are one
// member's level, which takes the partitioned line solve where part_eligible.
template <typename T>
void launch_smoother(const Problem &p, cudaStream_t s, const Lv<T> *L, const Item *it, int n,
                     double rho, int max_nz, int zero_mode, bool rows_ok, bool aligned,
                     int level);
bool rows_eligible(const Problem &p, int level);
// FP32 level whose line solves are partitioned (opts.line_part, small levels)
bool part_eligible(const Problem &p, int level);
bool restrict_rows_eligible(const Problem &p, int level);
bool restrict_rows_preferred(const Problem &p, int level);

ellsolve_status solve_ir(Plan &pl, const std::vector<const double *> &f,
                         const std::vector<double *> &x, double rtol, int maxit,
                         std::vector<ellsolve_result> &res);

}  // namespace ells

// The opaque handle of the C ABI is a Problem.
struct ellsolve_s : ells::Problem {};
