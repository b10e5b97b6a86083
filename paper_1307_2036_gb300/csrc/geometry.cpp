// Grid hierarchy for the periodic box and the cubed sphere (Sec. 3.1,
// Eqs. x1x2_1 / x1x2_2), with rediscretised coarse levels (Sec. 4.3.2: the
// coarse operators come from discretising on the coarse grid).
#include "geometry.hpp"

#include <cmath>
#include <stdexcept>

namespace ells {
namespace {

constexpr double kPi = 3.14159265358979323846;

struct Vec3 {
    double x, y, z;
};
inline Vec3 operator+(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline Vec3 operator*(double s, Vec3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline Vec3 cross(Vec3 a, Vec3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(Vec3 a) { return std::sqrt(dot(a, a)); }

// Cube faces: outward normal, then the directions of i and of j.
struct Frame {
    int nrm[3], ax[3], bx[3];
};
const Frame kFrames[6] = {
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},   {{0, 1, 0}, {-1, 0, 0}, {0, 0, 1}},
    {{-1, 0, 0}, {0, -1, 0}, {0, 0, 1}}, {{0, -1, 0}, {1, 0, 0}, {0, 0, 1}},
    {{0, 0, 1}, {0, 1, 0}, {-1, 0, 0}},  {{0, 0, -1}, {0, 1, 0}, {1, 0, 0}},
};

inline Vec3 v3(const int *a) { return {double(a[0]), double(a[1]), double(a[2])}; }
inline bool same(const int *a, const int *b) { return a[0] == b[0] && a[1] == b[1] && a[2] == b[2]; }
inline bool opposite(const int *a, const int *b) {
    return a[0] == -b[0] && a[1] == -b[1] && a[2] == -b[2];
}

// mapping coordinate (xi or eta) of grid position t in [0, n]
double map_coord(int mapping, double t, int n) {
    if (mapping == 1) return -1.0 + 2.0 * t / n;               // equidistant gnomonic
    return std::tan(-0.25 * kPi + 0.5 * kPi * t / n);          // equiangular
}

Vec3 on_sphere(int p, double xi, double eta) {
    const Frame &f = kFrames[p];
    Vec3 X = v3(f.nrm) + xi * v3(f.ax) + eta * v3(f.bx);
    return (1.0 / norm(X)) * X;
}

double arc(Vec3 a, Vec3 b) { return std::atan2(norm(cross(a, b)), dot(a, b)); }

// area of the gnomonic coordinate rectangle [x0,x1] x [y0,y1] on the unit
// sphere: F(x1,y1) - F(x0,y1) - F(x1,y0) + F(x0,y0), F = atan(xy / sqrt(1+x^2+y^2))
double gnomonic_area(double x0, double x1, double y0, double y1) {
    auto F = [](double x, double y) { return std::atan(x * y / std::sqrt(1.0 + x * x + y * y)); };
    return F(x1, y1) - F(x0, y1) - F(x1, y0) + F(x0, y0);
}

// Edge adjacency of the cube: for panel p and edge e (0 -i, 1 +i, 2 -j, 3 +j),
// the neighbouring panel, the edge of that panel touching p, and whether the
// running index along the edge is reversed.
struct EdgeLink {
    int panel, edge;
    bool reversed;
};

EdgeLink edge_link(int p, int e) {
    const Frame &f = kFrames[p];
    int out[3], run[3];
    const int *axis = (e < 2) ? f.ax : f.bx;
    const int *runax = (e < 2) ? f.bx : f.ax;
    int s = (e % 2 == 0) ? -1 : 1;
    for (int d = 0; d < 3; ++d) {
        out[d] = s * axis[d];
        run[d] = runax[d];
    }
    int q = -1;
    for (int c = 0; c < 6; ++c)
        if (same(kFrames[c].nrm, out)) q = c;
    const Frame &g = kFrames[q];
    // the edge of q that faces back towards p's normal direction
    int eq = -1;
    if (opposite(g.ax, f.nrm)) eq = 0;
    if (same(g.ax, f.nrm)) eq = 1;
    if (opposite(g.bx, f.nrm)) eq = 2;
    if (same(g.bx, f.nrm)) eq = 3;
    const int *qrun = (eq < 2) ? g.bx : g.ax;
    bool rev = opposite(qrun, run);
    if (q < 0 || eq < 0 || !(rev || same(qrun, run))) throw std::logic_error("cube edge table");
    return {q, eq, rev};
}

void build_box_level(HostLevel &L, int n, double side) {
    L.n = n;
    L.ncol = int64_t(n) * n;
    L.area.assign(L.ncol, 0.0);
    L.trans.assign(L.ncol * 4, 1.0);
    L.nbr.assign(L.ncol * 4, 0);
    const double h = side / n;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            int64_t c = int64_t(j) * n + i;
            L.area[c] = h * h;
            L.nbr[4 * c + 0] = int32_t(j * n + (i == 0 ? n - 1 : i - 1));
            L.nbr[4 * c + 1] = int32_t(j * n + (i == n - 1 ? 0 : i + 1));
            L.nbr[4 * c + 2] = int32_t((j == 0 ? n - 1 : j - 1) * n + i);
            L.nbr[4 * c + 3] = int32_t((j == n - 1 ? 0 : j + 1) * n + i);
        }
}

void build_sphere_level(HostLevel &L, int n, int mapping) {
    L.n = n;
    L.ncol = int64_t(6) * n * n;
    L.area.assign(L.ncol, 0.0);
    L.trans.assign(L.ncol * 4, 0.0);
    L.nbr.assign(L.ncol * 4, 0);
    std::vector<double> t(n + 1), tc(n);
    for (int a = 0; a <= n; ++a) t[a] = map_coord(mapping, a, n);
    for (int a = 0; a < n; ++a) tc[a] = map_coord(mapping, a + 0.5, n);

    EdgeLink links[6][4];
    for (int p = 0; p < 6; ++p)
        for (int e = 0; e < 4; ++e) links[p][e] = edge_link(p, e);

    auto index = [n](int p, int i, int j) { return (int64_t(p) * n + j) * n + i; };
    // neighbour across face e of cell (p, i, j)
    auto neighbour = [&](int p, int i, int j, int e) -> int64_t {
        int ii = i + (e == 0 ? -1 : e == 1 ? 1 : 0);
        int jj = j + (e == 2 ? -1 : e == 3 ? 1 : 0);
        if (ii >= 0 && ii < n && jj >= 0 && jj < n) return index(p, ii, jj);
        const EdgeLink &l = links[p][e];
        int run = (e < 2) ? j : i;
        if (l.reversed) run = n - 1 - run;
        switch (l.edge) {
            case 0: return index(l.panel, 0, run);
            case 1: return index(l.panel, n - 1, run);
            case 2: return index(l.panel, run, 0);
            default: return index(l.panel, run, n - 1);
        }
    };

    std::vector<Vec3> centre(L.ncol);
    for (int p = 0; p < 6; ++p)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) centre[index(p, i, j)] = on_sphere(p, tc[i], tc[j]);

    for (int p = 0; p < 6; ++p)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                int64_t c = index(p, i, j);
                L.area[c] = gnomonic_area(t[i], t[i + 1], t[j], t[j + 1]);
                Vec3 c00 = on_sphere(p, t[i], t[j]), c10 = on_sphere(p, t[i + 1], t[j]);
                Vec3 c01 = on_sphere(p, t[i], t[j + 1]), c11 = on_sphere(p, t[i + 1], t[j + 1]);
                const double face[4] = {arc(c00, c01), arc(c10, c11), arc(c00, c10), arc(c01, c11)};
                for (int e = 0; e < 4; ++e) {
                    int64_t q = neighbour(p, i, j, e);
                    L.nbr[4 * c + e] = int32_t(q);
                    L.trans[4 * c + e] = face[e] / arc(centre[c], centre[q]);
                }
            }
}

// Stencil of the cell-centred bilinear prolongation from level C (n/2) into
// level F (n): parent, the parent's neighbours towards the child in i and j,
// and the cell across the shared corner (-1 at a cube corner).
void build_prolongation(HostLevel &F, const HostLevel &C, int P) {
    const int nf = F.n, nc = C.n;
    const int64_t panel_cells = int64_t(nc) * nc;
    F.pst.assign(F.ncol * 4, -1);
    for (int p = 0; p < P; ++p)
        for (int j = 0; j < nf; ++j)
            for (int i = 0; i < nf; ++i) {
                int64_t f = (int64_t(p) * nf + j) * nf + i;
                int64_t par = (int64_t(p) * nc + j / 2) * nc + i / 2;
                int ex = (i & 1) ? 1 : 0, ey = (j & 1) ? 3 : 2;
                int64_t X = C.nbr[4 * par + ex], Y = C.nbr[4 * par + ey], D = -1;
                if (X / panel_cells == p) D = C.nbr[4 * X + ey];
                else if (Y / panel_cells == p) D = C.nbr[4 * Y + ex];
                F.pst[4 * f + 0] = int32_t(par);
                F.pst[4 * f + 1] = int32_t(X);
                F.pst[4 * f + 2] = int32_t(Y);
                F.pst[4 * f + 3] = int32_t(D);
            }
}

}  // namespace

HostHierarchy build_hierarchy(int kind, int n, int mapping, double side, int coarsest_min,
                              int max_levels) {
    if (n < 1) throw std::invalid_argument("n must be >= 1");
    HostHierarchy H;
    H.kind = kind;
    H.P = kind == 0 ? 1 : 6;
    H.mapping = mapping;
    H.side = side;
    int m = n;
    for (;;) {
        HostLevel L;
        if (kind == 0) build_box_level(L, m, side);
        else build_sphere_level(L, m, mapping);
        H.levels.push_back(std::move(L));
        if (m % 2 != 0 || m / 2 < coarsest_min) break;
        if (max_levels > 0 && int(H.levels.size()) >= max_levels) break;
        if (H.levels.size() >= 32) break;
        m /= 2;
    }
    for (size_t l = 0; l + 1 < H.levels.size(); ++l)
        build_prolongation(H.levels[l], H.levels[l + 1], H.P);
    return H;
}

void radial_vectors(const double *r, int nz, std::vector<double> &V, std::vector<double> &G) {
    V.assign(nz, 0.0);
    G.assign(nz + 1, 0.0);
    for (int k = 0; k < nz; ++k) {
        const double lo = r[k], hi = r[k + 1];
        // difference of cubes in factored form (thin cells keep full accuracy)
        V[k] = (hi - lo) * (hi * hi + hi * lo + lo * lo) / 3.0;
    }
    // rho_k - rho_{k-1} = (r_{k+1} - r_{k-1}) / 2
    for (int k = 1; k < nz; ++k) G[k] = 2.0 * r[k] * r[k] / (r[k + 1] - r[k - 1]);
}

}  // namespace ells
