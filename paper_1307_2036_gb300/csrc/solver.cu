// Host driver of the ellsolve C ABI: problem set-up, the multigrid V-cycle of
// Algorithm 1 as a fixed launch program over one or many problems, FP64
// multigrid, FP32-in-FP64 iterative refinement, and Algorithm PCG.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "ellsolve.h"
#include "geometry.hpp"
#include "kernels.hpp"
#include "solver.hpp"

namespace ells {

thread_local std::string t_last_error;

void set_last_error(const std::string &m) { t_last_error = m; }

void DevBuf::alloc(size_t b) {
    reset();
    if (b == 0) return;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        throw Error(e == cudaErrorMemoryAllocation ? ELLSOLVE_ERR_NOMEM : ELLSOLVE_ERR_CUDA,
                    "cudaMalloc(" + std::to_string(b) + " bytes): " + cudaGetErrorString(e));
    }
    bytes = b;
}

void DevBuf::reset() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

void check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(e == cudaErrorMemoryAllocation ? ELLSOLVE_ERR_NOMEM : ELLSOLVE_ERR_CUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
    }
}

template <typename T>
static void upload(DevBuf &d, const std::vector<T> &h, cudaStream_t s) {
    d.alloc(h.size() * sizeof(T));
    if (!h.empty()) {
        check_cuda(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s),
                   "upload");
        check_cuda(cudaStreamSynchronize(s), "upload sync");
    }
}

// ---------------------------------------------------------------------------
// Problem set-up
// ---------------------------------------------------------------------------
Problem::~Problem() {
    plan.reset();
    batch_plan.reset();
    if (pinned) cudaFreeHost(pinned);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (auto &e : ev_free) cudaEventDestroy(e);
    for (auto &e : ev_graph) cudaEventDestroy(e);
}

void Problem::build(const ellsolve_grid &g, double w2, double l2, const double *rl,
                    const ellsolve_opts &o, cudaStream_t s) {
    grid = g;
    opts = o;
    omega2 = w2;
    lambda2 = l2;
    stream = s;
    nz = g.nz;
    r.assign(rl, rl + nz + 1);
    HostHierarchy H = build_hierarchy(g.kind, g.n, g.mapping, g.box_side, o.coarsest_min,
                                      o.max_levels);
    P = H.P;
    nlev = int(H.levels.size());
    N = size_t(H.levels[0].ncol) * nz;

    std::vector<double> V, G;
    radial_vectors(r.data(), nz, V, G);
    std::vector<double> gv(nz + 1);
    for (int k = 0; k <= nz; ++k) gv[k] = w2 * l2 * G[k];
    std::vector<float> V32(V.begin(), V.end()), g32(gv.begin(), gv.end());
    upload(V64, V, s);
    upload(g64, gv, s);
    upload(this->V32, V32, s);
    upload(this->g32, g32, s);

    const bool need64 = true;                // level 0 always (outer residual, PCG)
    const bool need32 = o.precision == 1;
    lev.resize(nlev);
    h64.resize(nlev);
    h32.resize(nlev);
    for (int l = 0; l < nlev; ++l) {
        const HostLevel &hl = H.levels[l];
        LevelStore &L = lev[l];
        L.n = hl.n;
        L.ncol = int(hl.ncol);
        const size_t nc = size_t(hl.ncol), nl = nc * nz;
        std::vector<int4> nb(nc), ps(nc);
        for (size_t c = 0; c < nc; ++c) {
            nb[c] = make_int4(hl.nbr[4 * c], hl.nbr[4 * c + 1], hl.nbr[4 * c + 2], hl.nbr[4 * c + 3]);
            if (!hl.pst.empty())
                ps[c] = make_int4(hl.pst[4 * c], hl.pst[4 * c + 1], hl.pst[4 * c + 2], hl.pst[4 * c + 3]);
        }
        upload(L.nbr, nb, s);
        if (!hl.pst.empty()) upload(L.pst, ps, s);
        const bool lev64 = need64 && (l == 0 || o.precision == 0);
        if (lev64) {
            std::vector<double4_32a> tr(nc);
            for (size_t c = 0; c < nc; ++c)
                tr[c] = make_double4_32a(hl.trans[4 * c], hl.trans[4 * c + 1], hl.trans[4 * c + 2],
                                     hl.trans[4 * c + 3]);
            upload(L.area64, hl.area, s);
            upload(L.tr64, tr, s);
            if (o.precision == 0) {
                L.u64[0].alloc(nl * 8);
                L.u64[1].alloc(nl * 8);
                L.b64.alloc(nl * 8);
                L.aux64.alloc(nl * 8);
            }
        }
        if (need32) {
            std::vector<float> a32(hl.area.begin(), hl.area.end());
            std::vector<float4> tr(nc);
            for (size_t c = 0; c < nc; ++c)
                tr[c] = make_float4(float(hl.trans[4 * c]), float(hl.trans[4 * c + 1]),
                                    float(hl.trans[4 * c + 2]), float(hl.trans[4 * c + 3]));
            upload(L.area32, a32, s);
            upload(L.tr32, tr, s);
            L.u32[0].alloc(nl * 4);
            L.u32[1].alloc(nl * 4);
            L.b32.alloc(nl * 4);
            if (size_t(kBlk) * nz * 4 > 200 * 1024) L.aux32.alloc(nl * 4);
        }
        Lv<double> &d = h64[l];
        std::memset(&d, 0, sizeof(d));
        d.ncol = L.ncol;
        d.nz = nz;
        d.n = L.n;
        d.P = P;
        d.area = L.area64.as<double>();
        d.tr = L.tr64.as<double4_32a>();
        d.nbr = L.nbr.as<int4>();
        d.pst = L.pst.as<int4>();
        d.V = V64.as<double>();
        d.g = g64.as<double>();
        d.w2 = w2;
        d.u[0] = L.u64[0].as<double>();
        d.u[1] = L.u64[1].as<double>();
        d.b = L.b64.as<double>();
        d.aux = L.aux64.as<double>();
        Lv<float> &e = h32[l];
        std::memset(&e, 0, sizeof(e));
        e.ncol = L.ncol;
        e.nz = nz;
        e.n = L.n;
        e.P = P;
        e.area = L.area32.as<float>();
        e.tr = L.tr32.as<float4>();
        e.nbr = L.nbr.as<int4>();
        e.pst = L.pst.as<int4>();
        e.V = this->V32.as<float>();
        e.g = this->g32.as<float>();
        e.w2 = float(w2);
        e.u[0] = L.u32[0].as<float>();
        e.u[1] = L.u32[1].as<float>();
        e.b = L.b32.as<float>();
        e.aux = L.aux32.as<float>();
    }
    check_cuda(cudaHostAlloc(reinterpret_cast<void **>(&pinned), 64 * sizeof(double),
                             cudaHostAllocDefault),
               "cudaHostAlloc");
}

size_t Problem::footprint_bytes() const {
    size_t t = 0;
    for (const auto &L : lev)
        t += L.area64.bytes + L.tr64.bytes + L.area32.bytes + L.tr32.bytes + L.nbr.bytes +
             L.pst.bytes + L.u64[0].bytes + L.u64[1].bytes + L.b64.bytes + L.aux64.bytes +
             L.u32[0].bytes + L.u32[1].bytes + L.b32.bytes + L.aux32.bytes;
    return t;
}

// ---------------------------------------------------------------------------
// Plan: the launch program of a set of problems solved together
// ---------------------------------------------------------------------------
namespace {

struct MemberState {
    std::vector<int> cur;    // current ping-pong buffer per level
    std::vector<char> zero;  // level iterate known to be zero
};

void push_items(std::vector<Item> &v, int lv, int ncol, int in, int out, int zero) {
    for (int c0 = 0; c0 < ncol; c0 += kBlk) {
        Item it;
        it.lv = lv;
        it.col0 = c0;
        it.in = (unsigned char)in;
        it.out = (unsigned char)out;
        it.zero = (unsigned char)zero;
        it.pad = 0;
        v.push_back(it);
    }
}

}  // namespace

Plan::~Plan() { drop_graph(); }

void Plan::drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
}

void Plan::build(const std::vector<Problem *> &members, int prec) {
    mem = members;
    precision = prec;
    const int M = int(mem.size());
    base.assign(M, 0);
    int total = 0;
    maxlev = 0;
    maxnz = 0;
    for (int m = 0; m < M; ++m) {
        base[m] = total;
        total += mem[m]->nlev;
        maxlev = std::max(maxlev, mem[m]->nlev);
        maxnz = std::max(maxnz, mem[m]->nz);
    }
    cudaStream_t s = mem[0]->stream;
    std::vector<Lv<double>> d64;
    std::vector<Lv<float>> d32;
    for (int m = 0; m < M; ++m) {
        d64.insert(d64.end(), mem[m]->h64.begin(), mem[m]->h64.end());
        d32.insert(d32.end(), mem[m]->h32.begin(), mem[m]->h32.end());
    }
    upload(desc64, d64, s);
    upload(desc32, d32, s);
    items.clear();
    programs.clear();

    // items over the finest level of each member (outer kernels, lv = member)
    outer_first.assign(M + 1, 0);
    outer_off = 0;
    for (int m = 0; m < M; ++m) {
        outer_first[m] = int(items.size());
        push_items(items, m, mem[m]->lev[0].ncol, 0, 0, 0);
    }
    outer_first[M] = int(items.size());
    outer_n = int(items.size());
    // items over the finest level, lv = descriptor index, reading u[0] or u[1]
    for (int b = 0; b < 2; ++b) {
        norm_off[b] = int(items.size());
        for (int m = 0; m < M; ++m) push_items(items, base[m], mem[m]->lev[0].ncol, b, 0, 0);
        norm_n = int(items.size()) - norm_off[b];
    }

    std::vector<int> first_dev(outer_first.begin(), outer_first.end());
    upload(dfirst, first_dev, s);
    partials.alloc(size_t(std::max(outer_n, 1)) * sizeof(double));
    norms.alloc(size_t(M) * 4 * sizeof(double));
    scales.alloc(size_t(M) * sizeof(double));
    std::vector<double> cnt(M), ones(M, 1.0);
    for (int m = 0; m < M; ++m) cnt[m] = double(mem[m]->N);
    upload(counts, cnt, s);
    stage_active.assign(M, 1);
    upload(active, stage_active, s);
    check_cuda(cudaMemcpyAsync(scales.p, ones.data(), M * sizeof(double), cudaMemcpyHostToDevice, s),
               "scales");
    check_cuda(cudaStreamSynchronize(s), "plan sync");
    host_norms.assign(M, 0.0);
    items_dirty = true;
}

// Build the V-cycle program for the plan's members.  fine_zero: the finest
// iterate is zero on entry.  fine_cur: its buffer per member on entry.
const Program &Plan::program(bool fine_zero, const std::vector<int> &fine_cur) {
    std::string key = fine_zero ? "z" : "n";
    for (int c : fine_cur) key += char('0' + c);
    auto f = programs.find(key);
    if (f != programs.end()) return f->second;

    const Problem &p0 = *mem[0];
    const ellsolve_opts &o = p0.opts;
    const int M = int(mem.size());
    std::vector<MemberState> st(M);
    for (int m = 0; m < M; ++m) {
        st[m].cur.assign(mem[m]->nlev, 0);
        st[m].zero.assign(mem[m]->nlev, 1);
        st[m].cur[0] = fine_cur[m];
        st[m].zero[0] = fine_zero ? 1 : 0;
    }
    Program prog;
    auto lvl_count = [&](int m) { return mem[m]->nlev; };

    auto rows_level = [&](int m, int l) {
        const LevelStore &Ls = mem[m]->lev[l];
        return precision == 1 && Ls.n % 4 == 0 && Ls.ncol % 4 == 0 && mem[m]->nz % 8 == 0;
    };
    auto emit_smooth_one = [&](const std::vector<std::pair<int, int>> &ml, double rho) {
        if (ml.empty()) return;
        Op op;
        op.kind = Op::kSmooth;
        op.off = int(items.size());
        op.rho = rho;
        op.max_nz = 0;
        int nz_items = 0, z_items = 0;
        op.rows_ok = true;
        for (auto [m, l] : ml) {
            if (!rows_level(m, l)) op.rows_ok = false;
            MemberState &s = st[m];
            (s.zero[l] ? z_items : nz_items) += 1;
            push_items(items, base[m] + l, mem[m]->lev[l].ncol, s.cur[l], 1 - s.cur[l], s.zero[l]);
            s.cur[l] ^= 1;
            s.zero[l] = 0;
            op.max_nz = std::max(op.max_nz, mem[m]->nz);
            if (l == 0) {
                op.finest = true;
                const double w = precision == 1 ? 4.0 : 8.0;
                op.bytes += (items.back().zero ? 2.0 : 3.0) * w * double(mem[m]->N);
            }
        }
        op.n = int(items.size()) - op.off;
        op.zero_mode = z_items == 0 ? 0 : (nz_items == 0 ? 1 : 2);
        if (op.zero_mode == 2) op.rows_ok = false;
        prog.ops.push_back(op);
    };
    // one launch for the levels the row-staged kernel takes, one for the rest,
    // so that a member's kernel does not depend on the other members
    auto emit_smooth = [&](const std::vector<std::pair<int, int>> &ml, double rho) {
        std::vector<std::pair<int, int>> a, b;
        for (auto ml1 : ml) (rows_level(ml1.first, ml1.second) ? a : b).push_back(ml1);
        emit_smooth_one(a, rho);
        emit_smooth_one(b, rho);
    };
    auto emit_memsets = [&](const std::vector<std::pair<int, int>> &ml) {
        for (auto [m, l] : ml) {
            MemberState &s = st[m];
            if (!s.zero[l]) continue;
            Op op;
            op.kind = Op::kMemset;
            op.member = m;
            op.level = l;
            op.buf = s.cur[l];
            prog.ops.push_back(op);
            s.zero[l] = 0;
        }
    };

    // down the V: pre-smoothing and restriction, or the coarsest-level sweeps
    for (int d = 0; d < maxlev; ++d) {
        std::vector<std::pair<int, int>> pre, coarse;
        for (int m = 0; m < M; ++m) {
            if (d < lvl_count(m) - 1) pre.push_back({m, d});
            else if (d == lvl_count(m) - 1) coarse.push_back({m, d});
        }
        const int sweeps = std::max(pre.empty() ? 0 : o.nu_pre, coarse.empty() ? 0 : o.nu_coarse);
        for (int sw = 0; sw < sweeps; ++sw) {
            std::vector<std::pair<int, int>> a, b;
            if (sw < o.nu_pre) a = pre;
            if (sw < o.nu_coarse) b = coarse;
            emit_smooth(a, o.damping);
            emit_smooth(b, 1.0);
        }
        if (o.nu_coarse == 0) emit_memsets(coarse);
        if (!pre.empty()) {
            emit_memsets(pre);
            Op op;
            op.kind = Op::kRestrict;
            op.off = int(items.size());
            for (auto [m, l] : pre) {
                push_items(items, base[m] + l, mem[m]->lev[l + 1].ncol, st[m].cur[l], 0, 0);
                st[m].zero[l + 1] = 1;  // the coarse iterate starts from zero
                st[m].cur[l + 1] = 0;
            }
            op.n = int(items.size()) - op.off;
            prog.ops.push_back(op);
        }
    }
    // up the V: prolongation, correction and post-smoothing
    for (int d = maxlev - 2; d >= 0; --d) {
        std::vector<std::pair<int, int>> up;
        for (int m = 0; m < M; ++m)
            if (d < lvl_count(m) - 1) up.push_back({m, d});
        if (up.empty()) continue;
        Op op;
        op.kind = Op::kProlong;
        op.off = int(items.size());
        for (auto [m, l] : up)
            push_items(items, base[m] + l, mem[m]->lev[l].ncol, st[m].cur[l + 1], st[m].cur[l], 0);
        op.n = int(items.size()) - op.off;
        prog.ops.push_back(op);
        for (int sw = 0; sw < o.nu_post; ++sw) emit_smooth(up, o.damping);
    }
    prog.fine_cur_out.resize(M);
    for (int m = 0; m < M; ++m) prog.fine_cur_out[m] = st[m].cur[0];
    // items of the refinement update: read the correction from its final buffer
    prog.update_off = int(items.size());
    for (int m = 0; m < M; ++m) push_items(items, m, mem[m]->lev[0].ncol, st[m].cur[0], 0, 0);
    prog.update_n = int(items.size()) - prog.update_off;
    items_dirty = true;
    return programs.emplace(key, std::move(prog)).first->second;
}

void Plan::sync_items() {
    if (!items_dirty) return;
    cudaStream_t s = mem[0]->stream;
    upload(ditems, items, s);
    items_dirty = false;
    drop_graph();
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
static void count(Plan &pl, int n = 1) {
    for (Problem *p : pl.mem) p->launches += uint64_t(n);
}

template <typename T>
static const Lv<T> *descs(Plan &pl);
template <>
const Lv<double> *descs<double>(Plan &pl) { return pl.desc64.as<Lv<double>>(); }
template <>
const Lv<float> *descs<float>(Plan &pl) { return pl.desc32.as<Lv<float>>(); }

template <typename T>
static void run_program(Plan &pl, const Program &prog) {
    cudaStream_t s = pl.mem[0]->stream;
    const Item *it = pl.ditems.as<Item>();
    const Lv<T> *L = descs<T>(pl);
    const ellsolve_opts &o = pl.mem[0]->opts;
    Problem &p0 = *pl.mem[0];
    for (const Op &op : prog.ops) {
        switch (op.kind) {
            case Op::kSmooth: {
                const bool timed = p0.prof && op.finest;
                if (timed) p0.prof_mark_begin(s);
                if (sizeof(T) == 4 && op.rows_ok)
                    check_cuda(launch_smooth_rows(s, reinterpret_cast<const Lv<float> *>(L),
                                                  it + op.off, op.n, float(op.rho), op.max_nz,
                                                  op.zero_mode, p0.smooth_ctas_per_sm),
                               "smooth_rows");
                else
                    check_cuda(launch_smooth<T>(s, L, it + op.off, op.n, T(op.rho), op.max_nz,
                                                op.zero_mode),
                               "smooth");
                if (timed) p0.prof_mark_end(s, op.bytes);
                count(pl);
                break;
            }
            case Op::kRestrict:
                check_cuda(launch_restrict_resid<T>(s, L, it + op.off, op.n), "restrict");
                count(pl);
                break;
            case Op::kProlong:
                check_cuda(launch_prolong_add<T>(s, L, it + op.off, op.n, o.prolong), "prolong");
                count(pl);
                break;
            case Op::kMemset: {
                Problem &pm = *pl.mem[op.member];
                const LevelStore &Ls = pm.lev[op.level];
                const size_t bytes = size_t(Ls.ncol) * pm.nz * sizeof(T);
                void *ptr = sizeof(T) == 8 ? Ls.u64[op.buf].p : Ls.u32[op.buf].p;
                check_cuda(cudaMemsetAsync(ptr, 0, bytes, s), "memset");
                break;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Profiling of the finest-level smoother launches
// ---------------------------------------------------------------------------
// Outside a capture the pairs come from ev_free and are read after the next
// synchronisation; inside a capture they become event-record nodes of the
// graph (ev_graph) and are re-read after every replay.
void Problem::prof_mark_begin(cudaStream_t s) {
    std::vector<cudaEvent_t> &pool = capturing ? ev_graph : ev_free;
    int &next = capturing ? ev_graph_used : ev_next;
    while (next + 2 > int(pool.size())) {
        cudaEvent_t e;
        check_cuda(cudaEventCreate(&e), "cudaEventCreate");
        pool.push_back(e);
    }
    check_cuda(cudaEventRecordWithFlags(pool[next], s, capturing ? cudaEventRecordExternal : 0),
               "event record");
}

void Problem::prof_mark_end(cudaStream_t s, double bytes) {
    std::vector<cudaEvent_t> &pool = capturing ? ev_graph : ev_free;
    std::vector<double> &pb = capturing ? ev_graph_bytes : ev_free_bytes;
    int &next = capturing ? ev_graph_used : ev_next;
    check_cuda(cudaEventRecordWithFlags(pool[next + 1], s, capturing ? cudaEventRecordExternal : 0),
               "event record");
    if (int(pb.size()) < next / 2 + 1) pb.resize(next / 2 + 1);
    pb[next / 2] = bytes;
    next += 2;
}

void Problem::prof_collect(bool graph_replayed) {
    if (!prof) return;
    check_cuda(cudaStreamSynchronize(stream), "prof sync");
    auto read = [&](std::vector<cudaEvent_t> &pool, const std::vector<double> &pb, int used) {
        for (int i = 0; i + 1 < used; i += 2) {
            float ms = 0.f;
            check_cuda(cudaEventElapsedTime(&ms, pool[i], pool[i + 1]), "elapsed");
            prof_ms += ms;
            prof_bytes += pb[i / 2];
            prof_count += 1;
        }
    };
    read(ev_free, ev_free_bytes, ev_next);
    ev_next = 0;
    if (graph_replayed) read(ev_graph, ev_graph_bytes, ev_graph_used);
}

// ---------------------------------------------------------------------------
// Solvers
// ---------------------------------------------------------------------------
static double read_norms(Plan &pl, int M) {
    cudaStream_t s = pl.mem[0]->stream;
    double *h = pl.mem[0]->pinned;
    check_cuda(cudaMemcpyAsync(h, pl.norms.p, M * sizeof(double), cudaMemcpyDeviceToHost, s),
               "norm copy");
    check_cuda(cudaStreamSynchronize(s), "norm sync");
    for (int m = 0; m < M; ++m) pl.host_norms[m] = h[m];
    return h[0];
}

// Stagnation: no 10% reduction over the last 4 checks.
static bool stagnated(const std::vector<double> &hist) {
    const size_t n = hist.size();
    if (n < 5) return false;
    return hist[n - 1] > 0.9 * hist[n - 5];
}

static ellsolve_status finish(double rel, int it, double rtol, bool stag, ellsolve_result *res,
                              double secs) {
    if (res) {
        res->iterations = it;
        res->rel_residual = rel;
        res->seconds = secs;
    }
    if (!std::isfinite(rel)) {
        set_last_error("residual norm is not finite");
        return ELLSOLVE_ERR_NONFINITE;
    }
    (void)stag;
    return rel <= rtol ? ELLSOLVE_OK : ELLSOLVE_NOT_CONVERGED;
}

// One V-cycle of the FP64 hierarchy on the plan's members (fine iterate in
// u64[cur]).
static void vcycle64_once(Plan &pl, bool fine_zero) {
    std::vector<int> cur(pl.mem.size());
    for (size_t m = 0; m < pl.mem.size(); ++m) cur[m] = pl.mem[m]->fine_cur;
    const Program &prog = pl.program(fine_zero, cur);
    pl.sync_items();
    run_program<double>(pl, prog);
    for (size_t m = 0; m < pl.mem.size(); ++m) pl.mem[m]->fine_cur = prog.fine_cur_out[m];
}

// FP64 multigrid: b = vol f, u = 0, V-cycles until converged.
static ellsolve_status solve_mg64(Problem &p, const double *f, double *x, double rtol, int maxit,
                                  ellsolve_result *res) {
    Plan &pl = p.single_plan();
    cudaStream_t s = p.stream;
    auto t0 = std::chrono::steady_clock::now();
    pl.sync_items();
    check_cuda(launch_form_rhs<double>(s, pl.desc64.as<Lv<double>>(),
                                       pl.ditems.as<Item>() + pl.norm_off[0], pl.norm_n, f,
                                       p.h64[0].b, pl.partials.as<double>()),
               "form_rhs");
    check_cuda(launch_finalize(s, pl.partials.as<double>(), pl.dfirst.as<int>(), 1,
                               pl.norms.as<double>(), 1, nullptr, nullptr),
               "finalize");
    p.launches += 2;
    const double bnorm = read_norms(pl, 1);
    std::vector<double> hist{1.0};
    p.fine_cur = 0;
    double rel = bnorm > 0 ? 1.0 : 0.0;
    int iters = 0;
    bool stag = false;
    if (bnorm > 0) {
        for (iters = 1; iters <= maxit; ++iters) {
            vcycle64_once(pl, iters == 1);
            // residual norm of the fine iterate
            check_cuda(launch_resid<double>(s, pl.desc64.as<Lv<double>>(),
                                            pl.ditems.as<Item>() + pl.norm_off[p.fine_cur],
                                            pl.norm_n, 2, pl.partials.as<double>()),
                       "resid");
            check_cuda(launch_finalize(s, pl.partials.as<double>(), pl.dfirst.as<int>(), 1,
                                       pl.norms.as<double>(), 1, nullptr, nullptr),
                       "finalize");
            p.launches += 2;
            rel = read_norms(pl, 1) / bnorm;
            p.prof_collect(false);
            hist.push_back(rel);
            if (!(rel > rtol) || !std::isfinite(rel)) break;
            if (stagnated(hist)) {
                stag = true;
                break;
            }
        }
        if (iters > maxit) iters = maxit;
    }
    check_cuda(cudaMemcpyAsync(x, bnorm > 0 ? p.h64[0].u[p.fine_cur] : p.h64[0].b, p.N * 8,
                               cudaMemcpyDeviceToDevice, s),
               "copy out");
    if (bnorm == 0) check_cuda(cudaMemsetAsync(x, 0, p.N * 8, s), "zero x");
    check_cuda(cudaStreamSynchronize(s), "solve sync");
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return finish(rel, iters, rtol, stag, res, secs);
}

// Mixed precision: FP32 V-cycles on the FP64 residual (iterative refinement).
// The outer descriptors of each member point at its x and pointwise f.
static void ir_outer_descs(Plan &pl, const std::vector<const double *> &f,
                           const std::vector<double *> &x) {
    const int M = int(pl.mem.size());
    std::vector<Lv<double>> o64(M);
    std::vector<Lv<float>> f32(M);
    for (int m = 0; m < M; ++m) {
        o64[m] = pl.mem[m]->h64[0];
        o64[m].u[0] = x[m];
        o64[m].u[1] = nullptr;
        o64[m].b = const_cast<double *>(f[m]);
        f32[m] = pl.mem[m]->h32[0];
    }
    cudaStream_t s = pl.mem[0]->stream;
    if (pl.outer64.bytes != M * sizeof(Lv<double>)) pl.outer64.alloc(M * sizeof(Lv<double>));
    if (pl.fine32.bytes != M * sizeof(Lv<float>)) pl.fine32.alloc(M * sizeof(Lv<float>));
    // the host staging copy must outlive the asynchronous copy: keep it in the plan
    pl.stage64 = o64;
    pl.stage32 = f32;
    check_cuda(cudaMemcpyAsync(pl.outer64.p, pl.stage64.data(), M * sizeof(Lv<double>),
                               cudaMemcpyHostToDevice, s),
               "outer desc");
    check_cuda(cudaMemcpyAsync(pl.fine32.p, pl.stage32.data(), M * sizeof(Lv<float>),
                               cudaMemcpyHostToDevice, s),
               "fine desc");
    check_cuda(cudaStreamSynchronize(s), "desc sync");
    if (pl.gexec) {
        // descriptors changed in place; the graph reads them by address, so it stays valid
    }
}

static void ir_residual_norm(Plan &pl, int op, int x_is_zero = 0) {
    cudaStream_t s = pl.mem[0]->stream;
    const Item *it = pl.ditems.as<Item>();
    const int M = int(pl.mem.size());
    check_cuda(launch_ir_residual(s, pl.outer64.as<Lv<double>>(), pl.fine32.as<Lv<float>>(),
                                  it + pl.outer_off, pl.outer_n, pl.scales.as<double>(),
                                  pl.partials.as<double>(), x_is_zero),
               "ir_residual");
    check_cuda(launch_finalize(s, pl.partials.as<double>(), pl.dfirst.as<int>(), M,
                               pl.norms.as<double>(), op, op == 2 ? pl.scales.as<double>() : nullptr,
                               pl.counts.as<double>()),
               "finalize");
    count(pl, 2);
}

// one refinement step: inner V-cycles on r32, x += e / scale, new residual and norm
static void ir_step(Plan &pl) {
    cudaStream_t s = pl.mem[0]->stream;
    const int M = int(pl.mem.size());
    const int cycles = std::max(1, pl.mem[0]->opts.inner_cycles);
    std::vector<int> cur(M, 0);
    const Program *prog = &pl.program(true, cur);
    std::vector<const Program *> progs{prog};
    for (int c = 1; c < cycles; ++c) {
        prog = &pl.program(false, prog->fine_cur_out);
        progs.push_back(prog);
    }
    pl.sync_items();
    for (const Program *pr : progs) run_program<float>(pl, *pr);
    check_cuda(launch_ir_update(s, pl.outer64.as<Lv<double>>(), pl.fine32.as<Lv<float>>(),
                                pl.ditems.as<Item>() + progs.back()->update_off,
                                progs.back()->update_n, pl.scales.as<double>(),
                                pl.active.as<int>()),
               "ir_update");
    count(pl);
    ir_residual_norm(pl, 1);
}

static void ir_step_graph(Plan &pl) {
    Problem &p0 = *pl.mem[0];
    cudaStream_t s = p0.stream;
    // every program exists and the items are on the device before the capture
    {
        std::vector<int> cur(pl.mem.size(), 0);
        const Program *prog = &pl.program(true, cur);
        for (int c = 1; c < std::max(1, p0.opts.inner_cycles); ++c)
            prog = &pl.program(false, prog->fine_cur_out);
        pl.sync_items();
    }
    if (!pl.gexec) {
        // Capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph is launched on the
        // caller's stream below.
        if (!p0.cap_stream)
            check_cuda(cudaStreamCreateWithFlags(&p0.cap_stream, cudaStreamNonBlocking),
                       "capture stream");
        cudaStream_t cs = p0.cap_stream;
        for (Problem *p : pl.mem) {
            p->capturing = true;
            p->stream = cs;
        }
        auto restore = [&]() {
            for (Problem *p : pl.mem) {
                p->capturing = false;
                p->stream = s;
            }
        };
        const uint64_t before = p0.launches;
        p0.ev_graph_used = 0;
        check_cuda(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
        try {
            ir_step(pl);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            restore();
            throw;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t ec = cudaStreamEndCapture(cs, &graph);
        restore();
        check_cuda(ec, "end capture");
        cudaError_t e = cudaGraphInstantiate(&pl.gexec, graph, 0);
        cudaGraphDestroy(graph);
        check_cuda(e, "graph instantiate");
        pl.graph_launches = int(p0.launches - before);
        for (Problem *p : pl.mem) p->launches -= uint64_t(pl.graph_launches);
    }
    check_cuda(cudaGraphLaunch(pl.gexec, s), "graph launch");
    count(pl, pl.graph_launches);
}

ellsolve_status solve_ir(Plan &pl, const std::vector<const double *> &f,
                         const std::vector<double *> &x, double rtol, int maxit,
                         std::vector<ellsolve_result> &res) {
    const int M = int(pl.mem.size());
    Problem &p0 = *pl.mem[0];
    cudaStream_t s = p0.stream;
    auto t0 = std::chrono::steady_clock::now();
    for (int m = 0; m < M; ++m)
        check_cuda(cudaMemsetAsync(x[m], 0, pl.mem[m]->N * 8, s), "zero x");
    ir_outer_descs(pl, f, x);
    pl.sync_items();
    std::vector<double> ones(M, 1.0);
    pl.stage_scales = ones;
    check_cuda(cudaMemcpyAsync(pl.scales.p, pl.stage_scales.data(), M * sizeof(double),
                               cudaMemcpyHostToDevice, s),
               "scale reset");
    pl.stage_active.assign(M, 1);
    check_cuda(cudaMemcpyAsync(pl.active.p, pl.stage_active.data(), M * sizeof(int),
                               cudaMemcpyHostToDevice, s),
               "active reset");
    // ||b|| (x = 0 so the residual is b) and the FP32 scaling sqrt(N)/||b||
    ir_residual_norm(pl, 2, 1);
    read_norms(pl, M);
    std::vector<double> bnorm = pl.host_norms;
    // residual with the final scaling (x = 0 still)
    ir_residual_norm(pl, 1, 1);
    std::vector<std::vector<double>> hist(M, std::vector<double>{1.0});
    std::vector<int> iters(M, 0);
    std::vector<char> active(M, 1);
    std::vector<double> rel(M, 1.0);
    for (int m = 0; m < M; ++m)
        if (!(bnorm[m] > 0)) {
            active[m] = 0;
            rel[m] = 0.0;
        }
    const int cycles = std::max(1, p0.opts.inner_cycles);
    int step = 0;
    bool any = std::any_of(active.begin(), active.end(), [](char a) { return a != 0; });
    while (any && step * cycles < maxit) {
        if (p0.opts.use_graph) ir_step_graph(pl);
        else ir_step(pl);
        ++step;
        read_norms(pl, M);
        p0.prof_collect(p0.opts.use_graph != 0);
        for (int m = 0; m < M; ++m) {
            if (!active[m]) continue;
            iters[m] = step * cycles;
            rel[m] = pl.host_norms[m] / bnorm[m];
            hist[m].push_back(rel[m]);
            if (!(rel[m] > rtol) || !std::isfinite(rel[m]) || stagnated(hist[m])) active[m] = 0;
        }
        // A finished member rides along in the launches but its solution is
        // no longer updated, so it ends exactly where it would have alone.
        bool changed = false;
        for (int m = 0; m < M; ++m)
            if (pl.stage_active[m] != int(active[m])) {
                pl.stage_active[m] = active[m];
                changed = true;
            }
        if (changed)
            check_cuda(cudaMemcpyAsync(pl.active.p, pl.stage_active.data(), M * sizeof(int),
                                       cudaMemcpyHostToDevice, s),
                       "active");
        any = std::any_of(active.begin(), active.end(), [](char a) { return a != 0; });
    }
    check_cuda(cudaStreamSynchronize(s), "solve sync");
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    res.resize(M);
    ellsolve_status worst = ELLSOLVE_OK;
    for (int m = 0; m < M; ++m) {
        ellsolve_status st = finish(rel[m], iters[m], rtol, false, &res[m], secs);
        if (st < 0 || (st > worst && worst >= 0)) worst = st;
    }
    return worst;
}

// Algorithm PCG (FP64) with the block-Jacobi line preconditioner M = Dtilde.
static ellsolve_status solve_pcg(Problem &p, const double *f, double *x, double rtol, int maxit,
                                 ellsolve_result *res) {
    Plan &pl = p.single_plan();
    cudaStream_t s = p.stream;
    auto t0 = std::chrono::steady_clock::now();
    pl.sync_items();
    const size_t N = p.N;
    for (auto &b : p.cg)
        if (b.bytes != N * 8) b.alloc(N * 8);
    double *r = p.cg[0].as<double>(), *z = p.cg[1].as<double>(), *pp = p.cg[2].as<double>(),
           *q = p.cg[3].as<double>();
    if (p.cg_scal.bytes == 0) p.cg_scal.alloc(8 * sizeof(double));
    double *sc = p.cg_scal.as<double>();
    const Lv<double> *L = pl.desc64.as<Lv<double>>();
    const Item *it = pl.ditems.as<Item>() + pl.norm_off[0];
    const int ni = pl.norm_n;
    double *part = pl.partials.as<double>(), *nrm = pl.norms.as<double>();
    const int *first = pl.dfirst.as<int>();
    check_cuda(cudaMemsetAsync(x, 0, N * 8, s), "zero x");
    // r0 = b - A 0 = b
    check_cuda(launch_form_rhs<double>(s, L, it, ni, f, r, part), "form_rhs");
    check_cuda(launch_finalize(s, part, first, 1, nrm, 1, nullptr, nullptr), "finalize");
    const double r0 = read_norms(pl, 1);
    // z0 = M^-1 r0, kappa = <r0, z0>, p0 = z0
    check_cuda(launch_cg_precond_dot(s, L, it, ni, r, z, q, part), "precond");
    check_cuda(launch_finalize(s, part, first, 1, nrm + 1, 0, nullptr, nullptr), "finalize");
    check_cuda(launch_cg_scalars(s, sc, nrm + 1, 0), "scalars");
    check_cuda(cudaMemcpyAsync(pp, z, N * 8, cudaMemcpyDeviceToDevice, s), "p0");
    p.launches += 5;
    std::vector<double> hist{1.0};
    double rel = r0 > 0 ? 1.0 : 0.0;
    int K = 0;
    if (r0 > 0) {
        for (K = 1; K <= maxit; ++K) {
            check_cuda(launch_cg_apply_dot(s, L, it, ni, pp, q, part), "apply_dot");
            check_cuda(launch_finalize(s, part, first, 1, nrm + 1, 0, nullptr, nullptr), "fin");
            check_cuda(launch_cg_scalars(s, sc, nrm + 1, 1), "alpha");
            check_cuda(launch_cg_update(s, L, it, ni, x, r, pp, q, sc, part), "update");
            check_cuda(launch_finalize(s, part, first, 1, nrm, 1, nullptr, nullptr), "fin");
            p.launches += 5;
            rel = read_norms(pl, 1) / r0;
            hist.push_back(rel);
            if (rel < rtol || !std::isfinite(rel)) break;
            check_cuda(launch_cg_precond_dot(s, L, it, ni, r, z, q, part), "precond");
            check_cuda(launch_finalize(s, part, first, 1, nrm + 1, 0, nullptr, nullptr), "fin");
            check_cuda(launch_cg_scalars(s, sc, nrm + 1, 2), "beta");
            check_cuda(launch_cg_xpay(s, z, pp, sc, N), "xpay");
            p.launches += 4;
        }
        if (K > maxit) K = maxit;
    }
    check_cuda(cudaStreamSynchronize(s), "pcg sync");
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    // Algorithm PCG stops on the recursively updated residual; report it.
    return finish(rel, K, rtol, false, res, secs);
}

Plan &Problem::single_plan() {
    if (!plan) {
        plan = std::make_unique<Plan>();
        plan->build({this}, opts.precision);
    }
    return *plan;
}

// ---------------------------------------------------------------------------
// Level-API helper: a private descriptor pair with caller buffers
// ---------------------------------------------------------------------------
template <typename T>
struct LevelCall {
    DevBuf d;
    DevBuf it;
    std::vector<Lv<T>> h;
    std::vector<Item> items;
};

template <typename T>
static const std::vector<Lv<T>> &hdesc(const Problem &p);
template <>
const std::vector<Lv<double>> &hdesc<double>(const Problem &p) { return p.h64; }
template <>
const std::vector<Lv<float>> &hdesc<float>(const Problem &p) { return p.h32; }

template <typename T>
static ellsolve_status level_op(Problem &p, int level, int op, const void *a, const void *b,
                                void *out, int nsweeps, double rho) {
    if (level < 0 || level >= p.nlev) throw Error(ELLSOLVE_ERR_ARG, "level out of range");
    if (sizeof(T) == 8 && level > 0 && p.opts.precision != 0)
        throw Error(ELLSOLVE_ERR_ARG, "FP64 coarse levels exist only with precision 0");
    if (sizeof(T) == 4 && p.opts.precision != 1)
        throw Error(ELLSOLVE_ERR_ARG, "FP32 levels exist only with precision 1");
    const bool two = (op == 3 || op == 4);
    if (two && level + 1 >= p.nlev) throw Error(ELLSOLVE_ERR_ARG, "no coarser level");
    cudaStream_t s = p.stream;
    std::vector<Lv<T>> h;
    h.push_back(hdesc<T>(p)[level]);
    if (two) h.push_back(hdesc<T>(p)[level + 1]);
    const size_t nl = size_t(p.lev[level].ncol) * p.nz;
    DevBuf tmp;
    std::vector<Item> items;
    switch (op) {
        case 0:  // apply: aux = A u
            h[0].u[0] = static_cast<T *>(const_cast<void *>(a));
            h[0].aux = static_cast<T *>(out);
            push_items(items, 0, p.lev[level].ncol, 0, 0, 0);
            break;
        case 1:  // residual
            h[0].b = static_cast<T *>(const_cast<void *>(a));
            h[0].u[0] = static_cast<T *>(const_cast<void *>(b));
            h[0].aux = static_cast<T *>(out);
            push_items(items, 0, p.lev[level].ncol, 0, 0, 0);
            break;
        case 2: {  // smooth in place on out (= u), b = a; tmp = partner buffer + Thomas scratch
            tmp.alloc(2 * nl * sizeof(T));
            h[0].b = static_cast<T *>(const_cast<void *>(a));
            h[0].u[0] = static_cast<T *>(out);
            h[0].u[1] = tmp.as<T>();
            h[0].aux = tmp.as<T>() + nl;
            for (int sw = 0; sw < nsweeps; ++sw) push_items(items, 0, p.lev[level].ncol, sw & 1, 1 - (sw & 1), 0);
            break;
        }
        case 3:  // restrict residual: a = b, b = u, out = coarse b
            h[0].b = static_cast<T *>(const_cast<void *>(a));
            h[0].u[0] = static_cast<T *>(const_cast<void *>(b));
            h[1].b = static_cast<T *>(out);
            push_items(items, 0, p.lev[level + 1].ncol, 0, 0, 0);
            break;
        case 4:  // prolong add: a = coarse u, out = fine u
            h[1].u[0] = static_cast<T *>(const_cast<void *>(a));
            h[0].u[0] = static_cast<T *>(out);
            push_items(items, 0, p.lev[level].ncol, 0, 0, 0);
            break;
    }
    DevBuf dd, di;
    upload(dd, h, s);
    upload(di, items, s);
    const Lv<T> *L = dd.as<Lv<T>>();
    const Item *it = di.as<Item>();
    const int per = div_up(p.lev[level].ncol, kBlk);
    switch (op) {
        case 0: check_cuda(launch_resid<T>(s, L, it, per, 0, nullptr), "apply"); break;
        case 1: check_cuda(launch_resid<T>(s, L, it, per, 1, nullptr), "residual"); break;
        case 2: {
            const LevelStore &Ls = p.lev[level];
            const bool rows = sizeof(T) == 4 && Ls.n % 4 == 0 && Ls.ncol % 4 == 0 && p.nz % 8 == 0;
            for (int sw = 0; sw < nsweeps; ++sw) {
                if (rows)
                    check_cuda(launch_smooth_rows(s, reinterpret_cast<const Lv<float> *>(L),
                                                  it + sw * per, per, float(rho), p.nz, 0,
                                                  p.smooth_ctas_per_sm),
                               "smooth_rows");
                else
                    check_cuda(launch_smooth<T>(s, L, it + sw * per, per, T(rho), p.nz, 0), "smooth");
            }
            if (nsweeps & 1)
                check_cuda(cudaMemcpyAsync(out, tmp.p, nl * sizeof(T), cudaMemcpyDeviceToDevice, s),
                           "copy back");
            break;
        }
        case 3:
            check_cuda(launch_restrict_resid<T>(s, L, it, div_up(p.lev[level + 1].ncol, kBlk)),
                       "restrict");
            break;
        case 4: check_cuda(launch_prolong_add<T>(s, L, it, per, p.opts.prolong), "prolong"); break;
    }
    check_cuda(cudaStreamSynchronize(s), "level op sync");
    return ELLSOLVE_OK;
}

}  // namespace ells

// ===========================================================================
// C ABI
// ===========================================================================
using namespace ells;

#define ELLS_GUARD_BEGIN try {
#define ELLS_GUARD_END                                                   \
    }                                                                    \
    catch (const Error &e) {                                             \
        set_last_error(e.what());                                        \
        return e.status;                                                 \
    }                                                                    \
    catch (const std::bad_alloc &) {                                     \
        set_last_error("host allocation failed");                        \
        return ELLSOLVE_ERR_NOMEM;                                       \
    }                                                                    \
    catch (const std::exception &e) {                                    \
        set_last_error(e.what());                                        \
        return ELLSOLVE_ERR_ARG;                                         \
    }

extern "C" {

void ellsolve_default_opts(ellsolve_opts *o) {
    if (!o) return;
    o->precision = 0;
    o->solver = 0;
    o->nu_pre = 2;
    o->nu_post = 2;
    o->nu_coarse = 2;
    o->damping = 0.8;
    o->coarsest_min = 4;
    o->max_levels = 0;
    o->prolong = 0;
    o->inner_cycles = 1;
    o->use_graph = 1;
}

const char *ellsolve_last_error(void) { return t_last_error.c_str(); }

ellsolve_status ellsolve_create(const ellsolve_grid *grid, double omega2, double lambda2,
                                const double *r_levels, const ellsolve_opts *opts, void *stream,
                                ellsolve_t *out) {
    ELLS_GUARD_BEGIN
    if (!grid || !r_levels || !out) throw Error(ELLSOLVE_ERR_ARG, "null argument");
    *out = nullptr;
    if (grid->kind != 0 && grid->kind != 1) throw Error(ELLSOLVE_ERR_ARG, "grid.kind must be 0 or 1");
    if (grid->n < 1 || grid->nz < 1) throw Error(ELLSOLVE_ERR_ARG, "grid.n and grid.nz must be >= 1");
    if (grid->kind == 0 && !(grid->box_side > 0)) throw Error(ELLSOLVE_ERR_ARG, "box_side must be > 0");
    if (grid->kind == 1 && grid->mapping != 0 && grid->mapping != 1)
        throw Error(ELLSOLVE_ERR_ARG, "mapping must be 0 or 1");
    if (!(omega2 > 0) || !(lambda2 > 0)) throw Error(ELLSOLVE_ERR_ARG, "omega2 and lambda2 must be > 0");
    const size_t ncol = size_t(grid->kind == 0 ? 1 : 6) * grid->n * grid->n;
    if (ncol * size_t(grid->nz) >= (size_t(1) << 31))
        throw Error(ELLSOLVE_ERR_ARG, "more than 2^31 unknowns per problem");
    for (int k = 0; k < grid->nz; ++k)
        if (!(r_levels[k + 1] > r_levels[k])) throw Error(ELLSOLVE_ERR_ARG, "r_levels not increasing");
    ellsolve_opts o;
    ellsolve_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != 0 && o.precision != 1) throw Error(ELLSOLVE_ERR_ARG, "precision must be 0 or 1");
    if (o.solver != 0 && o.solver != 1) throw Error(ELLSOLVE_ERR_ARG, "solver must be 0 or 1");
    if (o.solver == 1 && o.precision != 0) throw Error(ELLSOLVE_ERR_ARG, "PCG runs in FP64 (precision 0)");
    if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_coarse < 0 || o.nu_pre + o.nu_post + o.nu_coarse == 0)
        throw Error(ELLSOLVE_ERR_ARG, "sweep counts must be >= 0 and not all zero");
    if (!(o.damping > 0 && o.damping <= 2)) throw Error(ELLSOLVE_ERR_ARG, "damping must be in (0, 2]");
    if (o.coarsest_min < 1) o.coarsest_min = 1;
    if (o.prolong != 0 && o.prolong != 1) throw Error(ELLSOLVE_ERR_ARG, "prolong must be 0 or 1");
    auto h = std::make_unique<ellsolve_s>();
    h->build(*grid, omega2, lambda2, r_levels, o, static_cast<cudaStream_t>(stream));
    *out = h.release();
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}

void ellsolve_destroy(ellsolve_t h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    delete h;
}

size_t ellsolve_size(ellsolve_t h) { return h ? h->N : 0; }
int ellsolve_num_levels(ellsolve_t h) { return h ? h->nlev : 0; }

ellsolve_status ellsolve_apply(ellsolve_t h, const void *x, void *y) {
    ELLS_GUARD_BEGIN
    if (!h || !x || !y) throw Error(ELLSOLVE_ERR_ARG, "null argument");
    return level_op<double>(*h, 0, 0, x, nullptr, y, 0, 0.0);
    ELLS_GUARD_END
}

ellsolve_status ellsolve_vcycle(ellsolve_t h, const void *f, void *u) {
    ELLS_GUARD_BEGIN
    if (!h || !f || !u) throw Error(ELLSOLVE_ERR_ARG, "null argument");
    Plan &pl = h->single_plan();
    cudaStream_t s = h->stream;
    if (h->opts.precision == 0) {
        pl.sync_items();
        const Item *it = pl.ditems.as<Item>();
        check_cuda(launch_form_rhs<double>(s, pl.desc64.as<Lv<double>>(), it + pl.norm_off[0],
                                           pl.norm_n, static_cast<const double *>(f), h->h64[0].b,
                                           pl.partials.as<double>()),
                   "form_rhs");
        check_cuda(cudaMemcpyAsync(h->h64[0].u[0], u, h->N * 8, cudaMemcpyDeviceToDevice, s), "in");
        h->fine_cur = 0;
        vcycle64_once(pl, false);
        check_cuda(cudaMemcpyAsync(u, h->h64[0].u[h->fine_cur], h->N * 8, cudaMemcpyDeviceToDevice, s),
                   "out");
    } else {
        std::vector<const double *> fv{static_cast<const double *>(f)};
        std::vector<double *> xv{static_cast<double *>(u)};
        ir_outer_descs(pl, fv, xv);
        pl.sync_items();
        // scaling from ||b||: residual of x = 0 would need a zero x, so scale by the current residual
        std::vector<double> ones(1, 1.0);
        pl.stage_scales = ones;
        check_cuda(cudaMemcpyAsync(pl.scales.p, pl.stage_scales.data(), sizeof(double),
                                   cudaMemcpyHostToDevice, s),
                   "scale");
        ir_residual_norm(pl, 2);
        ir_residual_norm(pl, 1);
        ir_step(pl);
    }
    check_cuda(cudaStreamSynchronize(s), "vcycle sync");
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}

ellsolve_status ellsolve_solve(ellsolve_t h, const void *rhs, void *x, double rtol, int maxit,
                               ellsolve_result *res) {
    ELLS_GUARD_BEGIN
    if (!h || !rhs || !x) throw Error(ELLSOLVE_ERR_ARG, "null argument");
    if (maxit < 0 || !(rtol >= 0)) throw Error(ELLSOLVE_ERR_ARG, "bad rtol or maxit");
    const double *f = static_cast<const double *>(rhs);
    double *xd = static_cast<double *>(x);
    if (h->opts.solver == 1) return solve_pcg(*h, f, xd, rtol, maxit, res);
    if (h->opts.precision == 0) return solve_mg64(*h, f, xd, rtol, maxit, res);
    Plan &pl = h->single_plan();
    std::vector<ellsolve_result> rr;
    ellsolve_status st = solve_ir(pl, {f}, {xd}, rtol, maxit, rr);
    if (res) *res = rr[0];
    return st;
    ELLS_GUARD_END
}

ellsolve_status ellsolve_solve_batch(ellsolve_t *handles, int count, const void *const *rhs,
                                     void *const *x, double rtol, int maxit, ellsolve_result *res) {
    ELLS_GUARD_BEGIN
    if (!handles || count <= 0 || !rhs || !x) throw Error(ELLSOLVE_ERR_ARG, "bad batch arguments");
    std::vector<Problem *> mem;
    std::vector<const double *> f;
    std::vector<double *> xv;
    for (int m = 0; m < count; ++m) {
        if (!handles[m] || !rhs[m] || !x[m]) throw Error(ELLSOLVE_ERR_ARG, "null member");
        if (handles[m]->opts.precision != 1 || handles[m]->opts.solver != 0)
            throw Error(ELLSOLVE_ERR_ARG, "batch members need precision 1 and solver 0");
        mem.push_back(handles[m]);
        f.push_back(static_cast<const double *>(rhs[m]));
        xv.push_back(static_cast<double *>(x[m]));
    }
    // one cached plan per member list (keyed on the first handle)
    Problem &p0 = *handles[0];
    if (!p0.batch_plan || p0.batch_plan->mem != mem) {
        p0.batch_plan = std::make_unique<Plan>();
        p0.batch_plan->build(mem, 1);
    }
    std::vector<ellsolve_result> rr;
    ellsolve_status st = solve_ir(*p0.batch_plan, f, xv, rtol, maxit, rr);
    if (res)
        for (int m = 0; m < count; ++m) res[m] = rr[m];
    return st;
    ELLS_GUARD_END
}

ellsolve_status ellsolve_level_shape(ellsolve_t h, int level, int *n, size_t *ncol) {
    ELLS_GUARD_BEGIN
    if (!h || level < 0 || level >= h->nlev) throw Error(ELLSOLVE_ERR_ARG, "bad level");
    if (n) *n = h->lev[level].n;
    if (ncol) *ncol = size_t(h->lev[level].ncol);
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}

#define LEVEL_DISPATCH(...) \
    (fp32 ? level_op<float>(*h, __VA_ARGS__) : level_op<double>(*h, __VA_ARGS__))

ellsolve_status ellsolve_level_apply(ellsolve_t h, int level, int fp32, const void *x, void *y) {
    ELLS_GUARD_BEGIN
    if (!h || !x || !y) throw Error(ELLSOLVE_ERR_ARG, "null argument");
    return LEVEL_DISPATCH(level, 0, x, nullptr, y, 0, 0.0);
    ELLS_GUARD_END
}

ellsolve_status ellsolve_level_residual(ellsolve_t h, int level, int fp32, const void *b,
                                        const void *u, void *r) {
    ELLS_GUARD_BEGIN
    if (!h || !b || !u || !r) throw Error(ELLSOLVE_ERR_ARG, "null argument");
    return LEVEL_DISPATCH(level, 1, b, u, r, 0, 0.0);
    ELLS_GUARD_END
}

ellsolve_status ellsolve_level_smooth(ellsolve_t h, int level, int fp32, const void *b, void *u,
                                      int nsweeps, double rho) {
    ELLS_GUARD_BEGIN
    if (!h || !b || !u || nsweeps < 0) throw Error(ELLSOLVE_ERR_ARG, "bad argument");
    if (nsweeps == 0) return ELLSOLVE_OK;
    return LEVEL_DISPATCH(level, 2, b, nullptr, u, nsweeps, rho);
    ELLS_GUARD_END
}

ellsolve_status ellsolve_level_restrict_residual(ellsolve_t h, int level, int fp32, const void *b,
                                                 const void *u, void *b_c) {
    ELLS_GUARD_BEGIN
    if (!h || !b || !u || !b_c) throw Error(ELLSOLVE_ERR_ARG, "null argument");
    return LEVEL_DISPATCH(level, 3, b, u, b_c, 0, 0.0);
    ELLS_GUARD_END
}

ellsolve_status ellsolve_level_prolong_add(ellsolve_t h, int level, int fp32, const void *u_c,
                                           void *u) {
    ELLS_GUARD_BEGIN
    if (!h || !u_c || !u) throw Error(ELLSOLVE_ERR_ARG, "null argument");
    return LEVEL_DISPATCH(level, 4, u_c, nullptr, u, 0, 0.0);
    ELLS_GUARD_END
}

ellsolve_status ellsolve_profile_enable(ellsolve_t h, int enable) {
    ELLS_GUARD_BEGIN
    if (!h) throw Error(ELLSOLVE_ERR_ARG, "null handle");
    h->prof = enable != 0;
    h->prof_ms = 0.0;
    h->prof_bytes = 0.0;
    h->prof_count = 0;
    h->ev_next = 0;
    if (h->plan) h->plan->drop_graph();
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}

ellsolve_status ellsolve_profile_read(ellsolve_t h, double *ms, int *launches, double *bytes) {
    ELLS_GUARD_BEGIN
    if (!h) throw Error(ELLSOLVE_ERR_ARG, "null handle");
    if (ms) *ms = h->prof_ms;
    if (launches) *launches = int(h->prof_count);
    if (bytes) *bytes = h->prof_bytes;
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}

uint64_t ellsolve_launch_count(ellsolve_t h) { return h ? h->launches : 0; }

}  // extern "C"
