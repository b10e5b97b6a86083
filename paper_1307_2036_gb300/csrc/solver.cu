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
#include <mutex>
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
    if (p && b <= cap) {
        bytes = b;
        return;
    }
    reset();
    if (b == 0) return;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        throw Error(e == cudaErrorMemoryAllocation ? ELLSOLVE_ERR_NOMEM : ELLSOLVE_ERR_CUDA,
                    "cudaMalloc(" + std::to_string(b) + " bytes): " + cudaGetErrorString(e));
    }
    bytes = cap = b;
}

void DevBuf::reset() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = cap = 0;
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
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (auto &e : ev_free) cudaEventDestroy(e);
    for (auto &e : ev_graph) cudaEventDestroy(e);
}

// ---------------------------------------------------------------------------
// Geometry cache
// ---------------------------------------------------------------------------
namespace {
struct GeoKey {
    int kind, n, mapping, cmin, maxl;
    double side;
    bool operator<(const GeoKey &o) const {
        if (kind != o.kind) return kind < o.kind;
        if (n != o.n) return n < o.n;
        if (mapping != o.mapping) return mapping < o.mapping;
        if (cmin != o.cmin) return cmin < o.cmin;
        if (maxl != o.maxl) return maxl < o.maxl;
        return side < o.side;
    }
};
std::mutex g_geo_mu;
std::map<GeoKey, std::weak_ptr<const Geometry>> g_geo_cache;

GeoKey geo_key(const ellsolve_grid &g, int coarsest_min, int max_levels) {
    return GeoKey{g.kind, g.n, g.kind == 1 ? g.mapping : 0, coarsest_min, max_levels,
                  g.kind == 0 ? g.box_side : 0.0};
}
}  // namespace

std::shared_ptr<const Geometry> geometry_for(const ellsolve_grid &g, int coarsest_min,
                                             int max_levels, cudaStream_t s) {
    const GeoKey key = geo_key(g, coarsest_min, max_levels);
    std::lock_guard<std::mutex> lock(g_geo_mu);
    auto f = g_geo_cache.find(key);
    if (f != g_geo_cache.end())
        if (auto sp = f->second.lock()) return sp;
    HostHierarchy H = build_hierarchy(g.kind, g.n, g.mapping, g.box_side, coarsest_min, max_levels);
    auto geo = std::make_shared<Geometry>();
    geo->kind = H.kind;
    geo->P = H.P;
    geo->mapping = H.mapping;
    geo->lev.resize(H.levels.size());
    for (size_t l = 0; l < H.levels.size(); ++l) {
        const HostLevel &hl = H.levels[l];
        LevelGeom &L = geo->lev[l];
        L.n = hl.n;
        L.ncol = int(hl.ncol);
        for (double ar : hl.area) L.area_sq += ar * ar;
        const size_t nc = size_t(hl.ncol);
        std::vector<int4> nb(nc), ps(nc);
        std::vector<double4_32a> tr64(nc);
        std::vector<float4> tr32(nc);
        std::vector<float> a32(hl.area.begin(), hl.area.end());
        for (size_t c = 0; c < nc; ++c) {
            nb[c] = make_int4(hl.nbr[4 * c], hl.nbr[4 * c + 1], hl.nbr[4 * c + 2], hl.nbr[4 * c + 3]);
            if (!hl.pst.empty())
                ps[c] = make_int4(hl.pst[4 * c], hl.pst[4 * c + 1], hl.pst[4 * c + 2], hl.pst[4 * c + 3]);
            const double *t = &hl.trans[4 * c];
            tr64[c] = make_double4_32a(t[0], t[1], t[2], t[3]);
            tr32[c] = make_float4(float(t[0]), float(t[1]), float(t[2]), float(t[3]));
        }
        upload(L.nbr, nb, s);
        if (!hl.pst.empty()) upload(L.pst, ps, s);
        upload(L.area64, hl.area, s);
        upload(L.tr64, tr64, s);
        upload(L.area32, a32, s);
        upload(L.tr32, tr32, s);
        geo->bytes += L.nbr.bytes + L.pst.bytes + L.area64.bytes + L.tr64.bytes + L.area32.bytes +
                      L.tr32.bytes;
    }
    std::shared_ptr<const Geometry> out = geo;
    g_geo_cache[key] = out;
    return out;
}

namespace {
// levels (n, ncol) of the hierarchy a grid gets, without building it
std::vector<std::pair<int, size_t>> level_sizes(const ellsolve_grid &g, const ellsolve_opts &o) {
    std::vector<std::pair<int, size_t>> v;
    const size_t P = g.kind == 0 ? 1 : 6;
    int m = g.n;
    for (;;) {
        v.push_back({m, P * size_t(m) * m});
        if (m % 2 != 0 || m / 2 < std::max(1, o.coarsest_min)) break;
        if (o.max_levels > 0 && int(v.size()) >= o.max_levels) break;
        if (v.size() >= 32) break;
        m /= 2;
    }
    return v;
}
}  // namespace

size_t problem_vector_bytes(const ellsolve_grid &g, const ellsolve_opts &o) {
    size_t t = 0;
    bool first = true;
    for (auto [n, nc] : level_sizes(g, o)) {
        const size_t nl = nc * size_t(g.nz);
        if (o.precision == 0) t += 4 * nl * 8;
        else {
            t += 3 * nl * 4;
            if (smooth_uses_global_scratch(g.nz, 4)) t += nl * 4;
            if (first) t += nl * 8;  // tracked refinement residual (double-float)
        }
        (void)n;
        (void)first;
        first = false;
    }
    return t + size_t(4) * (g.nz + 1) * 8;
}

size_t geometry_bytes(const ellsolve_grid &g, const ellsolve_opts &o) {
    size_t t = 0;
    for (auto [n, nc] : level_sizes(g, o)) t += nc * (16 + 16 + 8 + 32 + 4 + 16);
    return t;
}

// ---------------------------------------------------------------------------
// Problem set-up
// ---------------------------------------------------------------------------
void Problem::build(const ellsolve_grid &g, double w2, double l2, const double *rl,
                    const ellsolve_opts &o, cudaStream_t s, const double *pc, const double *qf) {
    grid = g;
    opts = o;
    stream = s;
    check_cuda(cudaGetDevice(&device), "cudaGetDevice");
    nz = g.nz;
    geom = geometry_for(g, o.coarsest_min, o.max_levels, s);
    P = geom->P;
    nlev = int(geom->lev.size());
    N = size_t(geom->lev[0].ncol) * nz;
    V64.alloc(nz * 8);
    g64.alloc((nz + 1) * 8);
    V32.alloc(nz * 4);
    g32.alloc((nz + 1) * 4);
    lev.resize(nlev);
    h64.resize(nlev);
    h32.resize(nlev);
    shape.assign(nlev, LevelShape{});
    const bool glob32 = smooth_uses_global_scratch(nz, 4);
    for (int l = 0; l < nlev; ++l) {
        const LevelGeom &G = geom->lev[l];
        LevelStore &L = lev[l];
        L.geo = &G;
        L.n = G.n;
        L.ncol = G.ncol;
        const size_t nl = size_t(G.ncol) * nz;
        if (o.precision == 0) {
            L.u64[0].alloc(nl * 8);
            L.u64[1].alloc(nl * 8);
            L.b64.alloc(nl * 8);
            L.aux64.alloc(nl * 8);
        } else {
            L.u32[0].alloc(nl * 4);
            L.u32[1].alloc(nl * 4);
            L.b32.alloc(nl * 4);
            if (glob32) L.aux32.alloc(nl * 4);
            // finest level: the scaled refinement residual as double-float pairs
            if (l == 0) L.aux64.alloc(nl * 8);
        }
        Lv<double> &d = h64[l];
        std::memset(&d, 0, sizeof(d));
        d.ncol = L.ncol;
        d.nz = nz;
        d.n = L.n;
        d.P = P;
        d.area = G.area64.as<double>();
        d.tr = G.tr64.as<double4_32a>();
        d.nbr = G.nbr.as<int4>();
        d.pst = G.pst.as<int4>();
        d.V = V64.as<double>();
        d.g = g64.as<double>();
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
        e.area = G.area32.as<float>();
        e.tr = G.tr32.as<float4>();
        e.nbr = G.nbr.as<int4>();
        e.pst = G.pst.as<int4>();
        e.V = V32.as<float>();
        e.g = g32.as<float>();
        e.u[0] = L.u32[0].as<float>();
        e.u[1] = L.u32[1].as<float>();
        e.b = L.b32.as<float>();
        e.aux = L.aux32.as<float>();
    }
    rebind(w2, l2, rl, pc, qf);
}

void Problem::rebind(double w2, double l2, const double *rl, const double *pc, const double *qf) {
    omega2 = w2;
    lambda2 = l2;
    r.assign(rl, rl + nz + 1);
    std::vector<double> V, G;
    radial_vectors(r.data(), nz, V, G);
    // vertical background profiles: V_k = int p r^2 dr, G_k carries p q
    if (pc) p_cell.assign(pc, pc + nz);
    else p_cell.clear();
    if (qf) q_face.assign(qf, qf + nz + 1);
    else q_face.clear();
    if (!p_cell.empty())
        for (int k = 0; k < nz; ++k) V[k] *= p_cell[k];
    if (!q_face.empty())
        for (int k = 1; k < nz; ++k) G[k] *= q_face[k];
    double vsq = 0.0;
    for (int k = 0; k < nz; ++k) vsq += V[k] * V[k];
    b_unit_norm = std::sqrt(geom->lev[0].area_sq * vsq);
    std::vector<double> gv(nz + 1);
    for (int k = 0; k <= nz; ++k) gv[k] = w2 * l2 * G[k];
    std::vector<float> V32h(V.begin(), V.end()), g32h(gv.begin(), gv.end());
    check_cuda(cudaMemcpyAsync(V64.p, V.data(), nz * 8, cudaMemcpyHostToDevice, stream), "V");
    check_cuda(cudaMemcpyAsync(g64.p, gv.data(), (nz + 1) * 8, cudaMemcpyHostToDevice, stream), "g");
    check_cuda(cudaMemcpyAsync(V32.p, V32h.data(), nz * 4, cudaMemcpyHostToDevice, stream), "V32");
    check_cuda(cudaMemcpyAsync(g32.p, g32h.data(), (nz + 1) * 4, cudaMemcpyHostToDevice, stream),
               "g32");
    check_cuda(cudaStreamSynchronize(stream), "rebind sync");
    for (auto &d : h64) d.w2 = w2;
    for (auto &e : h32) e.w2 = float(w2);
    plan.reset();  // descriptors changed
}

size_t Problem::footprint_bytes() const {
    size_t t = V64.bytes + g64.bytes + V32.bytes + g32.bytes;
    for (const auto &L : lev)
        t += L.u64[0].bytes + L.u64[1].bytes + L.b64.bytes + L.aux64.bytes + L.u32[0].bytes +
             L.u32[1].bytes + L.b32.bytes + L.aux32.bytes;
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

void push_items(std::vector<Item> &v, int lv, int ncol, int in, int out, int zero, int colour = 0) {
    for (int c0 = 0; c0 < ncol; c0 += kBlk) {
        Item it;
        it.lv = lv;
        it.col0 = c0;
        it.in = (unsigned char)in;
        it.out = (unsigned char)out;
        it.zero = (unsigned char)zero;
        it.colour = (unsigned char)colour;
        v.push_back(it);
    }
}

}  // namespace

Plan::~Plan() {
    drop_graph();
    if (hnorms) cudaFreeHost(hnorms);
}

void Plan::drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
}

// (Re)build for a set of members; the device buffers of an earlier build are
// reused where large enough.
void Plan::build(const std::vector<Problem *> &members, int prec) {
    drop_graph();
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
    partials2.alloc(size_t(std::max(outer_n, 1)) * sizeof(double));
    partials3.alloc(size_t(std::max(outer_n, 1)) * sizeof(double));
    norms.alloc(size_t(M) * 4 * sizeof(double));
    scales.alloc(size_t(2) * M * sizeof(double));
    std::vector<double> cnt(M), ones(M, 1.0);
    for (int m = 0; m < M; ++m) cnt[m] = double(mem[m]->N);
    upload(counts, cnt, s);
    stage_active.assign(M, 1);
    upload(active, stage_active, s);
    std::vector<double> ones2(2 * M, 1.0);
    check_cuda(cudaMemcpyAsync(scales.p, ones2.data(), 2 * M * sizeof(double),
                               cudaMemcpyHostToDevice, s),
               "scales");
    check_cuda(cudaStreamSynchronize(s), "plan sync");
    host_norms.assign(3 * M, 0.0);
    if (hnorms_n < size_t(4 * M)) {
        if (hnorms) cudaFreeHost(hnorms);
        hnorms = nullptr;
        check_cuda(cudaHostAlloc(reinterpret_cast<void **>(&hnorms), size_t(4 * M) * sizeof(double),
                                 cudaHostAllocMapped),
                   "pinned norms");
        check_cuda(cudaHostGetDevicePointer(reinterpret_cast<void **>(&hnorms_dev), hnorms, 0),
                   "mapped norms");
        hnorms_n = size_t(4 * M);
    }
    items_dirty = true;
}

// Build the V-cycle program for the plan's members.  fine_zero: the finest
// iterate is zero on entry.  fine_cur: its buffer per member on entry.
// With opts.fmg a cycle from a zero finest iterate is one full-multigrid cycle.
const Program &Plan::program(bool fine_zero, const std::vector<int> &fine_cur) {
    const bool fmg = fine_zero && mem[0]->opts.fmg != 0;
    std::string key = fmg ? "F" : (fine_zero ? "z" : "n");
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

    auto rows_level = [&](int m, int l) { return precision == 1 && rows_eligible(*mem[m], l); };
    auto part_level = [&](int m, int l) { return precision == 1 && part_eligible(*mem[m], l); };
    auto emit_smooth_one = [&](const std::vector<std::pair<int, int>> &ml, double rho,
                               int colour, bool part) {
        if (ml.empty()) return;
        Op op;
        op.kind = Op::kSmooth;
        op.part = part;
        op.off = int(items.size());
        op.rho = rho;
        op.max_nz = 0;
        op.tune = ml.front().second;
        int nz_items = 0, z_items = 0;
        op.rows_ok = true;
        op.aligned = true;
        for (auto [m, l] : ml) {
            if (!rows_level(m, l)) op.rows_ok = false;
            if (mem[m]->lev[l].n % 32 != 0) op.aligned = false;
            MemberState &s = st[m];
            (s.zero[l] ? z_items : nz_items) += 1;
            push_items(items, base[m] + l, mem[m]->lev[l].ncol, s.cur[l], 1 - s.cur[l], s.zero[l],
                       colour);
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
        if (op.zero_mode == 2 && !op.part) op.rows_ok = false;  // the partitioned kernel reads each item's flag
        prog.ops.push_back(op);
    };
    // One sweep: a launch for the levels that take the partitioned line solve,
    // one for the levels the row-staged kernel takes and one for the rest, so
    // that a member's kernel does not depend on the other members; members with the block red-black SOR smoother take two
    // half-sweeps (red, then black).
    // Members are grouped by (smoother, damping): each member sweeps with its
    // own relaxation parameter (the coarsest level undamped, rho = 1).
    auto emit_smooth = [&](const std::vector<std::pair<int, int>> &ml, bool coarsest) {
        std::vector<std::pair<int, std::pair<int, double>>> keyed;  // member index, key
        std::vector<std::pair<int, double>> keys;
        for (size_t i = 0; i < ml.size(); ++i) {
            const ellsolve_opts &mo = mem[ml[i].first]->opts;
            const std::pair<int, double> key{mo.smoother, coarsest ? 1.0 : mo.damping};
            if (std::find(keys.begin(), keys.end(), key) == keys.end()) keys.push_back(key);
            keyed.push_back({int(i), key});
        }
        for (const auto &key : keys) {
            std::vector<std::pair<int, int>> group;
            for (const auto &kv : keyed)
                if (kv.second == key) group.push_back(ml[kv.first]);
            const int passes = key.first == 1 ? 2 : 1;
            for (int pass = 0; pass < passes; ++pass) {
                const int colour = key.first == 1 ? pass + 1 : 0;
                std::vector<std::pair<int, int>> pt, a, b;
                for (auto ml1 : group)
                    (part_level(ml1.first, ml1.second)   ? pt
                     : rows_level(ml1.first, ml1.second) ? a
                                                         : b)
                        .push_back(ml1);
                emit_smooth_one(pt, key.second, colour, true);
                emit_smooth_one(a, key.second, colour, false);
                emit_smooth_one(b, key.second, colour, false);
            }
        }
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

    // prolongation onto level l of the listed members; onto_zero: the fine
    // iterate is zero and is overwritten by the interpolation
    auto emit_prolong = [&](const std::vector<std::pair<int, int>> &up, bool onto_zero) {
        Op op;
        op.kind = Op::kProlong;
        op.tune = up.empty() ? 0 : up.front().second;
        op.off = int(items.size());
        for (auto [m, l] : up) {
            push_items(items, base[m] + l, mem[m]->lev[l].ncol, st[m].cur[l + 1], st[m].cur[l],
                       onto_zero ? 1 : 0);
            st[m].zero[l] = 0;
        }
        op.n = int(items.size()) - op.off;
        prog.ops.push_back(op);
    };
    // One V-cycle from level top down to each member's coarsest level and back
    // (Algorithm 1), for the members flagged in `in`.
    auto emit_v = [&](int top, const std::vector<char> &in) {
        // down the V: pre-smoothing and restriction, or the coarsest-level sweeps
        for (int d = top; d < maxlev; ++d) {
            std::vector<std::pair<int, int>> pre, coarse;
            for (int m = 0; m < M; ++m) {
                if (!in[m]) continue;
                if (d < lvl_count(m) - 1) pre.push_back({m, d});
                else if (d == lvl_count(m) - 1) coarse.push_back({m, d});
            }
            const int sweeps =
                std::max(pre.empty() ? 0 : o.nu_pre, coarse.empty() ? 0 : o.nu_coarse);
            for (int sw = 0; sw < sweeps; ++sw) {
                std::vector<std::pair<int, int>> a, b;
                if (sw < o.nu_pre) a = pre;
                if (sw < o.nu_coarse) b = coarse;
                emit_smooth(a, false);
                emit_smooth(b, true);
            }
            if (o.nu_coarse == 0) emit_memsets(coarse);
            if (!pre.empty()) {
                emit_memsets(pre);
                // one launch for the levels the row-staged kernel takes, one for the rest
                std::vector<std::pair<int, int>> rows_pre, other_pre;
                for (auto ml : pre)
                    (precision == 1 && restrict_rows_preferred(*mem[ml.first], ml.second)
                         ? rows_pre
                         : other_pre)
                        .push_back(ml);
                for (int pass = 0; pass < 2; ++pass) {
                    const auto &list = pass == 0 ? rows_pre : other_pre;
                    if (list.empty()) continue;
                    Op op;
                    op.kind = Op::kRestrict;
                    op.rows_ok = pass == 0;
                    op.tune = list.front().second;
                    op.off = int(items.size());
                    for (auto [m, l] : list) {
                        push_items(items, base[m] + l, mem[m]->lev[l + 1].ncol, st[m].cur[l], 0,
                                   0);
                        st[m].zero[l + 1] = 1;  // the coarse iterate starts from zero
                        st[m].cur[l + 1] = 0;
                    }
                    op.n = int(items.size()) - op.off;
                    prog.ops.push_back(op);
                }
            }
        }
        // up the V: prolongation, correction and post-smoothing
        for (int d = maxlev - 2; d >= top; --d) {
            std::vector<std::pair<int, int>> up;
            for (int m = 0; m < M; ++m)
                if (in[m] && d < lvl_count(m) - 1) up.push_back({m, d});
            if (up.empty()) continue;
            emit_prolong(up, false);
            for (int sw = 0; sw < o.nu_post; ++sw) emit_smooth(up, false);
        }
    };

    if (!fmg) {
        emit_v(0, std::vector<char>(M, 1));
    } else {
        // Full multigrid (Sec. 4.3): the right-hand side restricted to every
        // level, the coarsest level smoothed from zero, then on each finer
        // level the interpolated coarse solution as the start of one V-cycle.
        for (int d = 0; d + 1 < maxlev; ++d) {
            Op op;
            op.kind = Op::kRestrictRhs;
            op.off = int(items.size());
            for (int m = 0; m < M; ++m) {
                if (d >= lvl_count(m) - 1) continue;
                push_items(items, base[m] + d, mem[m]->lev[d + 1].ncol, 0, 0, 0);
                st[m].zero[d + 1] = 1;
                st[m].cur[d + 1] = 0;
            }
            op.n = int(items.size()) - op.off;
            if (op.n > 0) prog.ops.push_back(op);
        }
        std::vector<std::pair<int, int>> coarse;
        for (int m = 0; m < M; ++m) coarse.push_back({m, lvl_count(m) - 1});
        for (int sw = 0; sw < o.nu_coarse; ++sw) emit_smooth(coarse, true);
        if (o.nu_coarse == 0) emit_memsets(coarse);
        for (int l = maxlev - 2; l >= 0; --l) {
            std::vector<char> in(M, 0);
            std::vector<std::pair<int, int>> up;
            for (int m = 0; m < M; ++m)
                if (l < lvl_count(m) - 1) {
                    in[m] = 1;
                    up.push_back({m, l});
                }
            if (up.empty()) continue;
            emit_prolong(up, true);
            emit_v(l, in);
        }
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
bool restrict_rows_eligible(const Problem &p, int level) {
    return level + 1 < p.nlev && p.lev[level].n % 64 == 0;
}

// The V-cycle takes the row-staged restriction where it fills the GPU (at
// least four column blocks per SM); smaller levels take the per-thread kernel
// split along the vertical, which is latency-bound for a shorter time.
bool restrict_rows_preferred(const Problem &p, int level) {
    return restrict_rows_eligible(p, level) && p.lev[level + 1].ncol >= 4 * 152 * kBlk;
}

// Levels the twisted FP32 smoother takes (every other level and the FP64
// path take the generic kernel).
bool rows_eligible(const Problem &p, int level) {
    const LevelStore &Ls = p.lev[level];
    if (Ls.n % 4 != 0 || Ls.ncol % 4 != 0) return false;
    return p.nz % 16 == 0 && smooth_tw_fits(p.nz, 8);
}

// Levels whose partitioned sweep fits one wave (two CTAs of 32 columns per
// SM): their sweeps wait on the elimination chain of a column, which the
// partitioned solve cuts.  On larger levels (6 x 64 x 64 and up) the
// streaming ring kernel is faster (C3 level 3: 24 against 30 us per sweep).
constexpr int kPartMaxCols = 2 * 152 * 32;

bool part_eligible(const Problem &p, int level) {
    return p.opts.precision == 1 && p.opts.line_part == 1 && rows_eligible(p, level) &&
           smooth_part_fits(p.nz) && p.lev[level].ncol <= kPartMaxCols;
}

template <typename T>
static void launch_smoother_op(const Problem &p, cudaStream_t s, const Lv<T> *L, const Item *it,
                               int n, double rho, int max_nz, int zero_mode, bool rows_ok,
                               bool aligned, int level, bool part) {
    if (sizeof(T) == 4 && part) {
        check_cuda(launch_smooth_part(s, reinterpret_cast<const Lv<float> *>(L), it, n,
                                      float(rho), max_nz),
                   "smooth_part");
    } else if (sizeof(T) == 4 && rows_ok && zero_mode != 2) {
        const Lv<float> *Lf = reinterpret_cast<const Lv<float> *>(L);
        const LevelShape &sh = p.level_shape(level);
        const bool stg = smooth_stg_fits(max_nz) && (sh.staged == 1 || (sh.staged == 0 && n < 152));
        if (stg)
            check_cuda(launch_smooth_stg(s, Lf, it, n, float(rho), max_nz, zero_mode),
                       "smooth_stg");
        else
            check_cuda(launch_smooth_tw(s, Lf, it, n, float(rho), max_nz, zero_mode, sh.ctas,
                                        sh.ring, aligned, sh.tmem),
                       "smooth_tw");
    } else {
        check_cuda(launch_smooth<T>(s, L, it, n, T(rho), max_nz, zero_mode), "smooth");
    }
}

template <typename T>
void launch_smoother(const Problem &p, cudaStream_t s, const Lv<T> *L, const Item *it, int n,
                     double rho, int max_nz, int zero_mode, bool rows_ok, bool aligned,
                     int level) {
    launch_smoother_op<T>(p, s, L, it, n, rho, max_nz, zero_mode, rows_ok, aligned, level,
                          sizeof(T) == 4 && rows_ok && part_eligible(p, level));
}
template void launch_smoother<float>(const Problem &, cudaStream_t, const Lv<float> *,
                                     const Item *, int, double, int, int, bool, bool, int);
template void launch_smoother<double>(const Problem &, cudaStream_t, const Lv<double> *,
                                      const Item *, int, double, int, int, bool, bool, int);
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
                launch_smoother_op<T>(p0, s, L, it + op.off, op.n, op.rho, op.max_nz, op.zero_mode,
                                      op.rows_ok, op.aligned, op.tune, op.part);
                if (timed) p0.prof_mark_end(s, op.bytes);
                count(pl);
                break;
            }
            case Op::kRestrict:
                if (sizeof(T) == 4 && op.rows_ok)
                    check_cuda(launch_restrict_rows(s, reinterpret_cast<const Lv<float> *>(L),
                                                    it + op.off, op.n),
                               "restrict_rows");
                else
                    check_cuda(launch_restrict_resid<T>(s, L, it + op.off, op.n, pl.maxnz,
                                                        p0.level_shape(op.tune).restrict_chunk),
                               "restrict");
                count(pl);
                break;
            case Op::kRestrictRhs:
                check_cuda(launch_restrict_rhs<T>(s, L, it + op.off, op.n), "restrict_rhs");
                count(pl);
                break;
            case Op::kProlong:
                check_cuda(launch_prolong_add<T>(s, L, it + op.off, op.n, o.prolong, pl.maxnz,
                                                 p0.level_shape(op.tune).prolong_chunk),
                           "prolong");
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
// The first `nvals` (<= 2 M) device norms into host_norms.  A kernel writes
// them into mapped pinned memory: a device-to-host cudaMemcpyAsync would queue
// behind whatever large transfer the caller has on the copy engines.
static double read_norms(Plan &pl, int nvals) {
    const int M = nvals;
    cudaStream_t s = pl.mem[0]->stream;
    double *h = pl.hnorms;
    check_cuda(launch_copy_doubles(s, pl.norms.as<double>(), pl.hnorms_dev, M), "norm copy");
    count(pl);
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
                              double secs, double err_est = -1.0) {
    if (res) {
        res->iterations = it;
        res->rel_residual = rel;
        res->seconds = secs;
        res->rel_error_est = err_est;
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
    // no V-cycle ran (zero right-hand side or maxit 0): the solution is the zero
    // start, not whatever the hierarchy holds
    if (bnorm > 0 && iters > 0)
        check_cuda(cudaMemcpyAsync(x, p.h64[0].u[p.fine_cur], p.N * 8, cudaMemcpyDeviceToDevice, s),
                   "copy out");
    else
        check_cuda(cudaMemsetAsync(x, 0, p.N * 8, s), "zero x");
    check_cuda(cudaStreamSynchronize(s), "solve sync");
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return finish(rel, iters, rtol, stag, res, secs);
}

// ---------------------------------------------------------------------------
// Mixed precision: FP32 V-cycles on the FP64 residual (iterative refinement).
// The inner right-hand side of member m is r * s_m with s_m a power of two
// near sqrt(N)/||r||: scaling by a power of two is exact, so the result does
// not depend on when s_m was chosen (alone or in a batch) -- it only keeps the
// FP32 values away from underflow.  The update reads the scale the residual was
// formed with (scale_cur); the new residual is formed with scale_next.
// ---------------------------------------------------------------------------
static double pow2_scale(double norm, size_t N) {
    if (!(norm > 0) || !std::isfinite(norm)) return 1.0;
    return std::ldexp(1.0, -std::ilogb(norm / std::sqrt(double(N))));
}

static void put_bytes(Plan &pl, void *dst, const void *src, size_t n) {
    const int k = launch_put_bytes(pl.mem[0]->stream, dst, src, n);
    if (k < 0) check_cuda(cudaGetLastError(), "put_bytes");
    count(pl, k);
}

// Outer descriptors: member m's finest FP64 level with u[0] = x_m, b = f_m.
void ir_bind(Plan &pl, const std::vector<MemberRun *> &run) {
    const int M = int(pl.mem.size());
    pl.stage64.resize(M);
    pl.stage32.resize(M);
    for (int m = 0; m < M; ++m) {
        pl.stage64[m] = pl.mem[m]->h64[0];
        pl.stage64[m].u[0] = run[m]->x;
        pl.stage64[m].u[1] = nullptr;
        pl.stage64[m].b = const_cast<double *>(run[m]->f);
        pl.stage32[m] = pl.mem[m]->h32[0];
    }
    cudaStream_t s = pl.mem[0]->stream;
    if (pl.outer64.bytes != M * sizeof(Lv<double>)) pl.outer64.alloc(M * sizeof(Lv<double>));
    if (pl.fine32.bytes != M * sizeof(Lv<float>)) pl.fine32.alloc(M * sizeof(Lv<float>));
    // through kernel parameters, not copies (see launch_put_bytes): a caller's
    // transfer in flight on the copy engine does not hold up the solve
    put_bytes(pl, pl.outer64.p, pl.stage64.data(), M * sizeof(Lv<double>));
    put_bytes(pl, pl.fine32.p, pl.stage32.data(), M * sizeof(Lv<float>));
}

static void ir_push_state(Plan &pl, const std::vector<MemberRun *> &run) {
    const int M = int(pl.mem.size());
    pl.stage_scales.resize(2 * M);
    pl.stage_active.resize(M);
    for (int m = 0; m < M; ++m) {
        pl.stage_scales[m] = run[m]->scale_cur;
        pl.stage_scales[M + m] = run[m]->scale_next;
        // 0 idle, 1 tracked, 2 FP64, 3 tracked with x = 0 (the first update writes x)
        const MemberRun &r = *run[m];
        pl.stage_active[m] = r.active ? (r.mode == 1 && r.x_zero ? 3 : r.mode) : 0;
    }
    put_bytes(pl, pl.scales.p, pl.stage_scales.data(), 2 * M * sizeof(double));
    put_bytes(pl, pl.active.p, pl.stage_active.data(), M * sizeof(int));
}

// FP64 residual of members [m0, m1) formed with scale_next, its norm (norms[m])
// and, for a general x, the magnitude || |A| |x| || (norms[M + m])
static void ir_residual_norm(Plan &pl, int m0, int m1, int x_is_zero) {
    cudaStream_t s = pl.mem[0]->stream;
    const int M = int(pl.mem.size());
    const int i0 = pl.outer_first[m0], i1 = pl.outer_first[m1];
    check_cuda(launch_ir_residual(s, pl.outer64.as<Lv<double>>(), pl.fine32.as<Lv<float>>(),
                                  pl.ditems.as<Item>() + pl.outer_off + i0, i1 - i0,
                                  pl.scales.as<double>() + M, pl.partials.as<double>() + i0,
                                  x_is_zero, nullptr, 0, pl.partials2.as<double>() + i0,
                                  pl.maxnz),
               "ir_residual");
    check_cuda(launch_finalize(s, pl.partials.as<double>(), pl.dfirst.as<int>() + m0, m1 - m0,
                               pl.norms.as<double>() + m0, 1, nullptr, nullptr),
               "finalize");
    count(pl, 2);
    if (x_is_zero == 0) {
        check_cuda(launch_finalize(s, pl.partials2.as<double>(), pl.dfirst.as<int>() + m0,
                                   m1 - m0, pl.norms.as<double>() + M + m0, 1, nullptr, nullptr),
                   "finalize");
        count(pl);
    }
}

// Rounding bounds of the refinement residual (2-norms, relative to the
// magnitudes || |A| |v| ||): an FP64 evaluation, and one double-float update
// (products and sums with binary32 halves, about 12 roundings of 2^-48 each).
constexpr double kErrFp64 = 0x1p-50;
constexpr double kErrTrack = 0x1p-44;
constexpr double kErrRound = 0x1p-52;  // the FP64 rounding of each update of x

// Start members [m0, m1): x = 0 unless keep_x, ||r||, scales, first residual.
void ir_start(Plan &pl, std::vector<MemberRun *> &run, int m0, int m1, bool keep_x) {
    if (m1 <= m0) return;
    cudaStream_t s = pl.mem[0]->stream;
    pl.sync_items();
    for (int m = m0; m < m1; ++m) {
        MemberRun &r = *run[m];
        // x = 0: a tracked member's first update writes x without reading it;
        // an FP64 member's update reads it, so it is cleared now
        r.x_zero = false;
        if (!keep_x) {
            if (pl.mem[m]->opts.refine == 1)
                check_cuda(cudaMemsetAsync(r.x, 0, pl.mem[m]->N * 8, s), "zero x");
            else
                r.x_zero = true;
        }
        // from x = 0 the residual is b: its first scale is the one that
        // normalises b for f = 1; with x given, 1 until its residual is known
        r.scale_cur = r.scale_next =
            keep_x ? 1.0 : pow2_scale(pl.mem[m]->b_unit_norm, pl.mem[m]->N);
        r.active = true;
        r.iters = 0;
        r.hist.assign(1, 1.0);
        r.dx_first = r.dx_prev = r.dx_last = 0.0;
    }
    ir_push_state(pl, run);
    // x = 0: b (in double-float, with that scale) and its norm in one pass;
    // x given: the norm of its residual first, which fixes the scale
    ir_residual_norm(pl, m0, m1, keep_x ? 0 : 1);
    read_norms(pl, int(pl.mem.size()));
    bool again = keep_x;
    for (int m = m0; m < m1; ++m) {
        MemberRun &r = *run[m];
        r.bnorm = pl.host_norms[m];
        r.rel = std::isfinite(r.bnorm) ? (r.bnorm > 0 ? 1.0 : 0.0) : r.bnorm;
        if (!(r.bnorm > 0) || !std::isfinite(r.bnorm)) r.active = false;
        const double sc = pow2_scale(r.bnorm, pl.mem[m]->N);
        // A power of two changes no bit of the result; only a right-hand side
        // whose magnitude puts the scaled b more than 2^20 from unit RMS (the
        // FP32 range margin) is formed again with its own scale.
        if (keep_x || (r.active && (sc > 0x1p20 * r.scale_cur || sc < 0x1p-20 * r.scale_cur))) {
            r.scale_cur = r.scale_next = sc;
            again = true;
        }
    }
    if (again) {
        ir_push_state(pl, run);
        ir_residual_norm(pl, m0, m1, keep_x ? 0 : 1);
        if (keep_x) read_norms(pl, 2 * int(pl.mem.size()));
    }
    const int M = int(pl.mem.size());
    for (int m = m0; m < m1; ++m) {
        MemberRun &r = *run[m];
        // the stored residual: b in double-float (x = 0), or an FP64 evaluation
        r.mode = pl.mem[m]->opts.refine == 1 ? 2 : 1;
        r.magx = keep_x ? pl.host_norms[M + m] : 0.0;
        r.errb = keep_x ? kErrFp64 * r.magx : 0x1p-45 * r.bnorm;
    }
}

// one refinement step: inner V-cycles on r32, x += e / scale_cur, new residual
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
    // The end of the step, per member by its mode: FP64 members update x and
    // recompute the residual; tracked members do both in one double-float
    // pass.  The update items run over each member's finest columns in member
    // order, as the outer items do, so the partial sums land in the same slots.
    const Item *ui = pl.ditems.as<Item>() + progs.back()->update_off;
    const int un = progs.back()->update_n;
    const Lv<double> *L64 = pl.outer64.as<Lv<double>>();
    const Lv<float> *L32 = pl.fine32.as<Lv<float>>();
    check_cuda(launch_ir_update(s, L64, L32, ui, un, pl.scales.as<double>(), pl.active.as<int>(),
                                2, pl.partials3.as<double>()),
               "ir_update");
    check_cuda(launch_ir_residual(s, L64, L32, ui, un, pl.scales.as<double>() + M,
                                  pl.partials.as<double>(), 0, pl.active.as<int>(), 2,
                                  pl.partials2.as<double>(), pl.maxnz),
               "ir_residual");
    bool fine_aligned = true;
    for (const Problem *p : pl.mem) fine_aligned = fine_aligned && p->lev[0].n % 32 == 0;
    check_cuda(launch_ir_track(s, L64, L32, ui, un, pl.scales.as<double>(), pl.active.as<int>(), M,
                               pl.maxnz, pl.partials.as<double>(), pl.partials2.as<double>(),
                               pl.partials3.as<double>(), fine_aligned),
               "ir_track");
    check_cuda(launch_finalize(s, pl.partials.as<double>(), pl.dfirst.as<int>(), M,
                               pl.norms.as<double>(), 1, nullptr, nullptr),
               "finalize");
    check_cuda(launch_finalize(s, pl.partials2.as<double>(), pl.dfirst.as<int>(), M,
                               pl.norms.as<double>() + M, 1, nullptr, nullptr),
               "finalize");
    check_cuda(launch_finalize(s, pl.partials3.as<double>(), pl.dfirst.as<int>(), M,
                               pl.norms.as<double>() + 2 * M, 1, nullptr, nullptr),
               "finalize");
    count(pl, 6);
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

// One refinement step for every member, then the per-member bookkeeping:
// convergence (rtol, maxit, stagnation, non-finite) and the next scale.
void ir_advance(Plan &pl, std::vector<MemberRun *> &run, bool use_graph) {
    const int M = int(pl.mem.size());
    Problem &p0 = *pl.mem[0];
    const int cycles = std::max(1, p0.opts.inner_cycles);
    ir_push_state(pl, run);
    if (use_graph) ir_step_graph(pl);
    else ir_step(pl);
    read_norms(pl, 3 * M);
    p0.prof_collect(use_graph);
    for (int m = 0; m < M; ++m) {
        MemberRun &r = *run[m];
        if (!r.active) continue;
        r.x_zero = false;  // the update wrote x
        r.dx_prev = r.dx_last;
        r.dx_last = pl.host_norms[2 * M + m];
        if (r.iters == 0) r.dx_first = r.dx_last;
    }
    // Error bounds of the stored residual.  A tracked member whose bound is
    // not below 0.1% of its residual (or whose residual is not finite) gets
    // the residual recomputed in FP64 -- it replaces the tracked one -- and
    // stays on the FP64 path for the rest of the solve.
    std::vector<int> redo;
    for (int m = 0; m < M; ++m) {
        MemberRun &r = *run[m];
        if (!r.active) continue;
        const double nrm = pl.host_norms[m], mag = pl.host_norms[M + m];
        if (r.mode == 1) {
            r.magx += mag;
            r.errb += kErrTrack * mag + kErrRound * r.magx;
            if (!(r.errb <= 1e-3 * nrm)) redo.push_back(m);
        } else {
            r.magx = mag;
            r.errb = kErrFp64 * mag;
        }
    }
    if (!redo.empty()) {
        for (int m : redo) ir_residual_norm(pl, m, m + 1, 0);
        read_norms(pl, 2 * M);
        for (int m : redo) {
            MemberRun &r = *run[m];
            r.mode = 2;
            r.magx = pl.host_norms[M + m];
            r.errb = kErrFp64 * r.magx;
        }
    }
    for (int m = 0; m < M; ++m) {
        MemberRun &r = *run[m];
        if (!r.active) continue;
        r.iters += cycles;
        r.rel = pl.host_norms[m] / r.bnorm;
        r.hist.push_back(r.rel);
        r.scale_cur = r.scale_next;
        r.scale_next = pow2_scale(pl.host_norms[m], pl.mem[m]->N);
        if (!(r.rel > r.rtol) || !std::isfinite(r.rel) || r.iters >= r.maxit || stagnated(r.hist))
            r.active = false;
    }
}

bool ir_zero_unwritten(Plan &pl, const std::vector<MemberRun *> &run) {
    bool any = false;
    for (size_t m = 0; m < run.size(); ++m) {
        MemberRun &r = *run[m];
        if (r.active || !r.x_zero) continue;
        check_cuda(cudaMemsetAsync(r.x, 0, pl.mem[m]->N * 8, pl.mem[0]->stream), "zero x");
        r.x_zero = false;
        any = true;
    }
    return any;
}

// Estimate of ||x* - x|| / ||x*|| for a refinement solve from x = 0.  If the
// last step contracts the error by q, the error left after its update dx_S is
// q / (1 - q) ||dx_S||, and ||x*|| is the first update to within the first
// step's contraction (x = dx_1 after one step).  The last step's error
// contraction is taken as its residual reduction r_S / r_{S-1}, scaled by how
// much more the error than the residual contracted in the step before: that
// step's error contraction is ||dx_S|| / ||dx_{S-1}|| (each update is about
// the error before its step), its residual reduction r_{S-1} / r_{S-2}.
// Residuals contract faster than errors, their smooth part being amplified
// most by A^{-1}, so the residual reduction alone underestimates.  With q
// near or above 1 (stagnation at the FP64 attainable residual) the last
// update is taken, times ten.  0 for a zero right-hand side; 1 when no step
// ran (x = 0).
static double error_estimate(const MemberRun &r) {
    if (r.bnorm == 0.0) return 0.0;
    if (r.hist.size() < 2 || !(r.dx_first > 0)) return 1.0;
    const size_t S = r.hist.size() - 1;  // steps done; hist[0] = 1
    double q = r.hist[S] / r.hist[S - 1];
    if (S >= 2 && r.dx_prev > 0 && r.hist[S - 1] > 0) {
        const double qe_prev = r.dx_last / r.dx_prev;
        const double qr_prev = r.hist[S - 1] / r.hist[S - 2];
        if (qr_prev > 0) q *= std::max(1.0, qe_prev / qr_prev);
    }
    const double ratio = r.dx_last / r.dx_first;
    if (!std::isfinite(q) || !std::isfinite(ratio)) return -1.0;
    return ratio * (q < 0.9 ? q / (1.0 - q) : 10.0);
}

ellsolve_status run_result(const MemberRun &r, double secs, ellsolve_result *res) {
    return finish(r.rel, r.iters, r.rtol, false, res, secs, error_estimate(r));
}

ellsolve_status solve_ir(Plan &pl, const std::vector<const double *> &f,
                         const std::vector<double *> &x, double rtol, int maxit,
                         std::vector<ellsolve_result> &res) {
    const int M = int(pl.mem.size());
    Problem &p0 = *pl.mem[0];
    cudaStream_t s = p0.stream;
    auto t0 = std::chrono::steady_clock::now();
    std::vector<MemberRun> runs(M);
    std::vector<MemberRun *> run(M);
    for (int m = 0; m < M; ++m) {
        runs[m].f = f[m];
        runs[m].x = x[m];
        runs[m].rtol = rtol;
        runs[m].maxit = maxit;
        run[m] = &runs[m];
    }
    ir_bind(pl, run);
    ir_start(pl, run, 0, M, false);
    auto any = [&]() {
        return std::any_of(runs.begin(), runs.end(), [](const MemberRun &r) { return r.active; });
    };
    if (maxit <= 0)
        for (auto &r : runs) r.active = false;
    while (any()) ir_advance(pl, run, p0.opts.use_graph != 0);
    ir_zero_unwritten(pl, run);
    check_cuda(cudaStreamSynchronize(s), "solve sync");
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    res.resize(M);
    ellsolve_status worst = ELLSOLVE_OK;
    for (int m = 0; m < M; ++m) {
        ellsolve_status st = run_result(runs[m], secs, &res[m]);
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
    // the V-cycle preconditioner's program and items exist before any item
    // pointer is taken (building them may move the item buffer)
    const bool mgpc = p.opts.precond == 2;
    if (mgpc) {
        pl.program(true, std::vector<int>(1, 0));
        pl.sync_items();
    }
    const Lv<double> *L = pl.desc64.as<Lv<double>>();
    const Item *it = pl.ditems.as<Item>() + pl.norm_off[0];
    const int ni = pl.norm_n;
    double *part = pl.partials.as<double>(), *nrm = pl.norms.as<double>();
    const int *first = pl.dfirst.as<int>();
    check_cuda(cudaMemsetAsync(x, 0, N * 8, s), "zero x");
    // The preconditioner: block Jacobi z = Dtilde^{-1} r (one fused kernel
    // with <r, z>), or block red-black SSOR (Sec. 7.2): half-sweeps red,
    // black, black, red of A z = r from z = 0 with rho = 1 (symmetric block
    // Gauss-Seidel), on the FP64 level-0 buffers the solver does not use
    // otherwise, then <r, z>.
    const bool ssor = p.opts.precond == 1;
    DevBuf sdesc, sitems;
    const int per0 = div_up(p.lev[0].ncol, kBlk);
    if (ssor) {
        std::vector<Lv<double>> hd{p.h64[0]};
        hd[0].b = r;
        hd[0].u[0] = z;
        hd[0].u[1] = p.lev[0].u64[1].as<double>();
        hd[0].aux = p.lev[0].aux64.as<double>();
        std::vector<Item> items;
        const int seq[4][3] = {{0, 1, 1}, {1, 0, 2}, {0, 1, 2}, {1, 0, 1}};  // in, out, colour
        for (int h = 0; h < 4; ++h)
            push_items(items, 0, p.lev[0].ncol, seq[h][0], seq[h][1], h == 0 ? 1 : 0, seq[h][2]);
        upload(sdesc, hd, s);
        upload(sitems, items, s);
    }
    auto precond_dot = [&]() {
        if (mgpc) {
            // one FP64 V-cycle of A z = r from z = 0 on the multigrid hierarchy
            check_cuda(cudaMemcpyAsync(p.h64[0].b, r, N * 8, cudaMemcpyDeviceToDevice, s), "r");
            p.fine_cur = 0;
            vcycle64_once(pl, true);
            check_cuda(cudaMemcpyAsync(z, p.h64[0].u[p.fine_cur], N * 8, cudaMemcpyDeviceToDevice,
                                       s),
                       "z");
            check_cuda(launch_dot(s, L, it, ni, r, z, part), "dot");
            p.launches += 1;
        } else if (ssor) {
            for (int h = 0; h < 4; ++h)
                launch_smoother<double>(p, s, sdesc.as<Lv<double>>(), sitems.as<Item>() + h * per0,
                                        per0, 1.0, p.nz, h == 0 ? 1 : 0, false, false, 0);
            check_cuda(launch_dot(s, L, it, ni, r, z, part), "dot");
            p.launches += 4;
        } else {
            check_cuda(launch_cg_precond_dot(s, L, it, ni, r, z, q, part), "precond");
        }
    };
    // r0 = b - A 0 = b
    check_cuda(launch_form_rhs<double>(s, L, it, ni, f, r, part), "form_rhs");
    check_cuda(launch_finalize(s, part, first, 1, nrm, 1, nullptr, nullptr), "finalize");
    const double r0 = read_norms(pl, 1);
    // z0 = M^-1 r0, kappa = <r0, z0>, p0 = z0
    precond_dot();
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
            if (mgpc) {
                // the V-cycle is not a symmetric operator: flexible (Polak-Ribiere)
                // beta = (<r, z> - <r, z_old>) / kappa_old
                check_cuda(launch_dot(s, L, it, ni, r, z, part), "dot");
                check_cuda(launch_finalize(s, part, first, 1, nrm + 2, 0, nullptr, nullptr), "fin");
                p.launches += 2;
            }
            precond_dot();
            check_cuda(launch_finalize(s, part, first, 1, nrm + 1, 0, nullptr, nullptr), "fin");
            check_cuda(launch_cg_scalars(s, sc, nrm + 1, mgpc ? 3 : 2), "beta");
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
            // block red-black SOR: two half-sweeps per sweep, red then black
            const int launches = p.opts.smoother == 1 ? 2 * nsweeps : nsweeps;
            for (int sw = 0; sw < launches; ++sw)
                push_items(items, 0, p.lev[level].ncol, sw & 1, 1 - (sw & 1), 0,
                           p.opts.smoother == 1 ? 1 + (sw & 1) : 0);
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
            const bool rows = sizeof(T) == 4 && rows_eligible(p, level);
            const int launches = p.opts.smoother == 1 ? 2 * nsweeps : nsweeps;
            for (int sw = 0; sw < launches; ++sw)
                launch_smoother<T>(p, s, L, it + sw * per, per, rho, p.nz, 0, rows,
                                   p.lev[level].n % 32 == 0, level);
            if (launches & 1)
                check_cuda(cudaMemcpyAsync(out, tmp.p, nl * sizeof(T), cudaMemcpyDeviceToDevice, s),
                           "copy back");
            break;
        }
        case 3:
            if (sizeof(T) == 4 && restrict_rows_eligible(p, level))
                check_cuda(launch_restrict_rows(s, reinterpret_cast<const Lv<float> *>(L), it,
                                                div_up(p.lev[level + 1].ncol, kBlk)),
                           "restrict_rows");
            else
                check_cuda(launch_restrict_resid<T>(s, L, it, div_up(p.lev[level + 1].ncol, kBlk), p.nz,
                                                    p.level_shape(level).restrict_chunk),
                           "restrict");
            break;
        case 4:
            check_cuda(launch_prolong_add<T>(s, L, it, per, p.opts.prolong, p.nz,
                                             p.level_shape(level).prolong_chunk),
                       "prolong");
            break;
    }
    check_cuda(cudaStreamSynchronize(s), "level op sync");
    return ELLSOLVE_OK;
}

// Time `run` (one launch sequence) after a warm-up: the median of seven runs,
// each between its own pair of events, so that a gap in which the GPU waits
// for the host (a short launch enqueued late) or a disturbance of one run
// does not decide the choice.
template <typename F>
double time_ms(cudaStream_t s, cudaEvent_t, cudaEvent_t, F run) {
    constexpr int reps = 7;
    cudaEvent_t ev[2 * reps] = {};
    double t[reps];
    try {
        for (auto &e : ev) check_cuda(cudaEventCreate(&e), "event");
        run();
        for (int r = 0; r < reps; ++r) {
            check_cuda(cudaEventRecord(ev[2 * r], s), "record");
            run();
            check_cuda(cudaEventRecord(ev[2 * r + 1], s), "record");
        }
        check_cuda(cudaEventSynchronize(ev[2 * reps - 1]), "sync");
        for (int r = 0; r < reps; ++r) {
            float ms = 0.f;
            check_cuda(cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]), "elapsed");
            t[r] = ms;
        }
    } catch (...) {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
        throw;
    }
    for (auto e : ev) cudaEventDestroy(e);
    std::sort(t, t + reps);
    return t[reps / 2];
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
    o->inner_cycles = 3;
    o->use_graph = 1;
    o->smoother = 0;
    o->precond = 0;
    o->fmg = 0;
    o->refine = 0;
    o->line_part = 1;
}

const char *ellsolve_last_error(void) { return t_last_error.c_str(); }

ellsolve_status ellsolve_create(const ellsolve_grid *grid, double omega2, double lambda2,
                                const double *r_levels, const ellsolve_opts *opts, void *stream,
                                ellsolve_t *out) {
    return ellsolve_create_profiles(grid, omega2, lambda2, r_levels, nullptr, nullptr, opts,
                                    stream, out);
}

ellsolve_status ellsolve_create_profiles(const ellsolve_grid *grid, double omega2, double lambda2,
                                         const double *r_levels, const double *p_cell,
                                         const double *q_face, const ellsolve_opts *opts,
                                         void *stream, ellsolve_t *out) {
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
    if (p_cell)
        for (int k = 0; k < grid->nz; ++k)
            if (!(p_cell[k] > 0) || !std::isfinite(p_cell[k]))
                throw Error(ELLSOLVE_ERR_ARG, "p_cell must be positive and finite");
    if (q_face)
        for (int k = 1; k < grid->nz; ++k)
            if (!(q_face[k] > 0) || !std::isfinite(q_face[k]))
                throw Error(ELLSOLVE_ERR_ARG, "q_face must be positive and finite at 1..nz-1");
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
    if (o.smoother != 0 && o.smoother != 1) throw Error(ELLSOLVE_ERR_ARG, "smoother must be 0 or 1");
    if (o.precond < 0 || o.precond > 2) throw Error(ELLSOLVE_ERR_ARG, "precond must be 0, 1 or 2");
    if (o.fmg != 0 && o.fmg != 1) throw Error(ELLSOLVE_ERR_ARG, "fmg must be 0 or 1");
    if (o.refine != 0 && o.refine != 1) throw Error(ELLSOLVE_ERR_ARG, "refine must be 0 or 1");
    auto h = std::make_unique<ellsolve_s>();
    h->build(*grid, omega2, lambda2, r_levels, o, static_cast<cudaStream_t>(stream), p_cell, q_face);
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
        MemberRun r;
        r.f = static_cast<const double *>(f);
        r.x = static_cast<double *>(u);
        r.rtol = 0.0;
        r.maxit = 1;
        std::vector<MemberRun *> run{&r};
        ir_bind(pl, run);
        ir_start(pl, run, 0, 1, true);  // residual of the given iterate
        if (r.active) ir_advance(pl, run, false);
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
        // the launch sequence is shared: members may differ in grid, parameters,
        // smoother and damping, not in sweep counts, prolongation or schedule
        const ellsolve_opts &a = handles[m]->opts, &z = handles[0]->opts;
        if (a.nu_pre != z.nu_pre || a.nu_post != z.nu_post || a.nu_coarse != z.nu_coarse ||
            a.prolong != z.prolong || a.inner_cycles != z.inner_cycles || a.fmg != z.fmg)
            throw Error(ELLSOLVE_ERR_ARG,
                        "batch members need equal nu_pre, nu_post, nu_coarse, prolong, inner_cycles, fmg");
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

ellsolve_status ellsolve_autotune(ellsolve_t h, int *out_ctas, double *out_ms) {
    ELLS_GUARD_BEGIN
    if (!h) throw Error(ELLSOLVE_ERR_ARG, "null handle");
    if (h->opts.precision != 1) throw Error(ELLSOLVE_ERR_ARG, "autotune needs precision 1");
    cudaStream_t s = h->stream;
    cudaEvent_t e0, e1;
    check_cuda(cudaEventCreate(&e0), "event");
    check_cuda(cudaEventCreate(&e1), "event");
    double ms0 = 0.0;
    try {
        for (int l = 0; l < h->nlev; ++l) {
            using ells::time_ms;
            const LevelStore &Ls = h->lev[l];
            const size_t nl = size_t(Ls.ncol) * h->nz;
            const int nitems = div_up(Ls.ncol, kBlk);
            // the level's own FP32 buffers as scratch (zeroed)
            check_cuda(cudaMemsetAsync(Ls.u32[0].p, 0, nl * 4, s), "zero");
            check_cuda(cudaMemsetAsync(Ls.u32[1].p, 0, nl * 4, s), "zero");
            check_cuda(cudaMemsetAsync(Ls.b32.p, 0, nl * 4, s), "zero");
            std::vector<Lv<float>> hd{h->h32[l]};
            if (l + 1 < h->nlev) hd.push_back(h->h32[l + 1]);
            std::vector<Item> items;
            push_items(items, 0, Ls.ncol, 0, 1, 0);
            const int off_c = int(items.size());
            if (l + 1 < h->nlev) push_items(items, 0, h->lev[l + 1].ncol, 0, 0, 0);
            DevBuf dd, di;
            upload(dd, hd, s);
            upload(di, items, s);
            LevelShape &sh = h->shape[size_t(l)];
            // (a) the line smoother: resident CTAs per SM, ring depth and where
            // f' is parked, on the levels the twisted kernel takes
            if (rows_eligible(*h, l) && !part_eligible(*h, l)) {
                std::vector<LevelShape> cand;  // (ctas, ring, tmem, staged)
                const bool tm_ok = h->nz <= 256;
                const bool stg_ok = smooth_stg_fits(h->nz);
                if (nitems >= 152) {
                    for (int c : {3, 4, 5}) cand.push_back({c, 8, 0, 2});
                    cand.push_back({4, 4, 0, 2});
                    for (int c : {4, 5}) cand.push_back({c, 8, 2, 2});
                    cand.push_back({5, 4, 2, 2});
                    if (stg_ok && nitems < 4 * 152) cand.push_back({4, 8, 0, 1});
                } else {
                    if (stg_ok) cand.push_back({4, 8, 0, 1});
                    cand.push_back({4, 8, 2, 2});
                    cand.push_back({4, 4, 2, 2});
                    if (tm_ok) cand.push_back({4, 8, 1, 2});
                }
                double best = 1e300;
                LevelShape keep = sh;
                for (const LevelShape &c : cand) {
                    sh.ctas = c.ctas;
                    sh.ring = c.ring;
                    sh.tmem = c.tmem;
                    sh.staged = c.staged;
                    const double ms = time_ms(s, e0, e1, [&] {
                        launch_smoother<float>(*h, s, dd.as<Lv<float>>(), di.as<Item>(), nitems,
                                               0.8, h->nz, 0, true, Ls.n % 32 == 0, l);
                    });
                    if (ms < best) {
                        best = ms;
                        keep = sh;
                    }
                }
                sh.ctas = keep.ctas;
                sh.ring = keep.ring;
                sh.tmem = keep.tmem;
                sh.staged = keep.staged;
                if (l == 0) ms0 = best;
            } else if (l == 0 && part_eligible(*h, l)) {
                // the partitioned line solve has no launch shape: its time only
                ms0 = time_ms(s, e0, e1, [&] {
                    launch_smoother<float>(*h, s, dd.as<Lv<float>>(), di.as<Item>(), nitems, 0.8,
                                           h->nz, 0, true, Ls.n % 32 == 0, l);
                });
            }
            // (b) the transfers of small levels: how far to split them along
            // the vertical (the row-staged restriction of large levels is not
            // split)
            if (l + 1 < h->nlev) {
                const int nc_items = div_up(h->lev[l + 1].ncol, kBlk);
                const bool rows_r = restrict_rows_eligible(*h, l) && restrict_rows_preferred(*h, l);
                if (!rows_r && nc_items < 4 * 152) {
                    double best = 1e300;
                    int keep = sh.restrict_chunk;
                    for (int want : {152, 304, 608, 1216}) {
                        const double ms = time_ms(s, e0, e1, [&] {
                            check_cuda(launch_restrict_resid<float>(s, dd.as<Lv<float>>(),
                                                                    di.as<Item>() + off_c,
                                                                    nc_items, h->nz, want),
                                       "restrict");
                        });
                        if (ms < best) {
                            best = ms;
                            keep = want;
                        }
                    }
                    sh.restrict_chunk = keep;
                }
                if (nitems < 4 * 152) {
                    double best = 1e300;
                    int keep = sh.prolong_chunk;
                    for (int want : {152, 304, 608, 1216}) {
                        const double ms = time_ms(s, e0, e1, [&] {
                            check_cuda(launch_prolong_add<float>(s, dd.as<Lv<float>>(),
                                                                 di.as<Item>(), nitems,
                                                                 h->opts.prolong, h->nz, want),
                                       "prolong");
                        });
                        if (ms < best) {
                            best = ms;
                            keep = want;
                        }
                    }
                    sh.prolong_chunk = keep;
                }
            }
            check_cuda(cudaStreamSynchronize(s), "autotune sync");
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (h->plan) h->plan->drop_graph();
    if (h->batch_plan) h->batch_plan->drop_graph();
    if (out_ctas) *out_ctas = h->shape[0].ctas;
    if (out_ms) *out_ms = ms0;
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}
ellsolve_status ellsolve_selftest(uint64_t samples, uint64_t *mismatches) {
    ELLS_GUARD_BEGIN
    DevBuf bad;
    bad.alloc(sizeof(unsigned long long));
    check_cuda(cudaMemset(bad.p, 0, sizeof(unsigned long long)), "memset");
    check_cuda(launch_selftest_conv(0, samples, static_cast<unsigned long long *>(bad.p)),
               "selftest");
    unsigned long long h = 0;
    check_cuda(cudaMemcpy(&h, bad.p, sizeof(h), cudaMemcpyDeviceToHost), "selftest copy");
    if (mismatches) *mismatches = h;
    if (h != 0) throw Error(ELLSOLVE_ERR_CUDA, "conversion self-test: " + std::to_string(h) +
                                                   " mismatches");
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}

ellsolve_status ellsolve_set_tuning(ellsolve_t h, int ctas_per_sm, int ring) {
    ELLS_GUARD_BEGIN
    if (!h) throw Error(ELLSOLVE_ERR_ARG, "null handle");
    if (ctas_per_sm < 0 || ctas_per_sm > 16) throw Error(ELLSOLVE_ERR_ARG, "ctas_per_sm must be 0..16");
    if (ring != 4 && ring != 8) throw Error(ELLSOLVE_ERR_ARG, "ring must be 4 or 8");
    for (LevelShape &sh : h->shape) {
        sh.ctas = ctas_per_sm;
        sh.ring = ring;
    }
    if (h->plan) h->plan->drop_graph();
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}

ellsolve_status ellsolve_get_tuning(ellsolve_t h, int *ctas_per_sm, int *ring) {
    ELLS_GUARD_BEGIN
    if (!h) throw Error(ELLSOLVE_ERR_ARG, "null handle");
    if (ctas_per_sm) *ctas_per_sm = h->shape[0].ctas;
    if (ring) *ring = h->shape[0].ring;
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}

ellsolve_status ellsolve_set_level_tuning(ellsolve_t h, int level, int ctas_per_sm, int ring,
                                          int tmem, int staged, int restrict_chunk,
                                          int prolong_chunk) {
    ELLS_GUARD_BEGIN
    if (!h || level < 0 || level >= h->nlev) throw Error(ELLSOLVE_ERR_ARG, "bad handle or level");
    if (ctas_per_sm < 0 || ctas_per_sm > 16) throw Error(ELLSOLVE_ERR_ARG, "ctas_per_sm must be 0..16");
    if (ring != 4 && ring != 8) throw Error(ELLSOLVE_ERR_ARG, "ring must be 4 or 8");
    if (tmem < 0 || tmem > 2) throw Error(ELLSOLVE_ERR_ARG, "tmem must be 0, 1 or 2");
    if (staged < 0 || staged > 2) throw Error(ELLSOLVE_ERR_ARG, "staged must be 0, 1 or 2");
    if (restrict_chunk < 1 || prolong_chunk < 1)
        throw Error(ELLSOLVE_ERR_ARG, "chunk targets must be >= 1");
    LevelShape &sh = h->shape[size_t(level)];
    sh.ctas = ctas_per_sm;
    sh.ring = ring;
    sh.tmem = tmem;
    sh.staged = staged;
    sh.restrict_chunk = restrict_chunk;
    sh.prolong_chunk = prolong_chunk;
    if (h->plan) h->plan->drop_graph();
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}

ellsolve_status ellsolve_get_level_tuning(ellsolve_t h, int level, int *ctas_per_sm, int *ring,
                                          int *tmem, int *staged, int *restrict_chunk,
                                          int *prolong_chunk) {
    ELLS_GUARD_BEGIN
    if (!h || level < 0 || level >= h->nlev) throw Error(ELLSOLVE_ERR_ARG, "bad handle or level");
    const LevelShape &sh = h->shape[size_t(level)];
    if (ctas_per_sm) *ctas_per_sm = sh.ctas;
    if (ring) *ring = sh.ring;
    if (tmem) *tmem = sh.tmem;
    if (staged) *staged = sh.staged;
    if (restrict_chunk) *restrict_chunk = sh.restrict_chunk;
    if (prolong_chunk) *prolong_chunk = sh.prolong_chunk;
    return ELLSOLVE_OK;
    ELLS_GUARD_END
}

}  // extern "C"
