// Host-side set-up of the WQ library: mesh topology and classification, the
// bicubic unstructured spline space in Bezier form, the exactness-set pattern
// and the min-max point counts.
//
// Paper: Sheng, Wei, Chen, "Weighted Quadrature on Unstructured Splines".
//   Sec. 3  terminology (valence, EP, irregular/enriched/transition/boundary/
//           passive elements), mesh assumptions (no EP in the boundary 1-ring,
//           knot spans 1 except 0 across edges perpendicular to the boundary),
//           the analysis space (vertex-based bicubic B-splines, four face-based
//           C1 double-knot B-splines per enriched face, truncation, EP splines
//           eliminated, 2x2 split + D-patch in irregular faces, Fig. 2).
//   Table 1 function counts per element type (reproduced by this construction).
//   Eq. 10  exactness set S_i; Sec. 4.2 Eq. qp_allocation (min-max counts).
//
// Construction (each function = its control variable set to 1, all others 0):
//   inner Bezier points of a face: the face DOF at that corner if the face is
//     enriched, else the span-ratio division of the face's 4 vertex DOFs;
//   edge points: span-weighted mean of the two inner points across the edge;
//   corner points: tensor span-weighted mean of the 4 inner points around a
//     valence-4 vertex, plain mean of the mu inner points around an EP;
//   irregular faces: de Casteljau split at 1/2; around every EP the sub-net at
//     the EP gets d10 = d01 = d00 (collapsed), spoke points d20 projected onto
//     the first Fourier mode around the EP and d11 = mean of its two spoke
//     points (coplanar).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>
#include <unordered_set>

#include "wq_internal.h"

namespace wqi {

static const double COEF_TOL = 1e-12;
static const int CU[4] = {0, 1, 1, 0};
static const int CV[4] = {0, 0, 1, 1};

// ---------------------------------------------------------------- topology
bool build_topology(const wq_mesh_desc& mesh, Topology& T, Error& err) {
    const int64_t V = mesh.n_vertices, F = mesh.n_faces;
    T.V = V;
    T.F = F;
    T.quads.assign(mesh.quads, mesh.quads + 4 * F);
    for (int64_t f = 0; f < F; ++f) {
        for (int c = 0; c < 4; ++c) {
            int32_t v = T.quads[f * 4 + c];
            if (v < 0 || v >= V) {
                err = {WQ_ERR_MESH, "face " + std::to_string(f) + " has a vertex id out of range"};
                return false;
            }
            for (int d = 0; d < c; ++d)
                if (T.quads[f * 4 + d] == v) {
                    err = {WQ_ERR_MESH, "face " + std::to_string(f) + " repeats a vertex"};
                    return false;
                }
        }
    }
    // edges: (min, max, face, k) sorted
    struct Ed { int32_t a, b; int32_t f; int8_t k; };
    std::vector<Ed> ed(4 * F);
    for (int64_t f = 0; f < F; ++f)
        for (int k = 0; k < 4; ++k) {
            int32_t a = T.quads[f * 4 + k], b = T.quads[f * 4 + (k + 1) % 4];
            ed[f * 4 + k] = {std::min(a, b), std::max(a, b), (int32_t)f, (int8_t)k};
        }
    std::sort(ed.begin(), ed.end(), [](const Ed& x, const Ed& y) {
        return x.a != y.a ? x.a < y.a : (x.b != y.b ? x.b < y.b : x.f < y.f);
    });
    T.nb_face.assign(4 * F, -1);
    T.nb_edge.assign(4 * F, -1);
    T.bnd_vertex.assign(V, 0);
    std::vector<std::vector<int32_t>> nbr(V);
    for (size_t i = 0; i < ed.size();) {
        size_t j = i;
        while (j < ed.size() && ed[j].a == ed[i].a && ed[j].b == ed[i].b) ++j;
        size_t cnt = j - i;
        if (cnt > 2) {
            err = {WQ_ERR_MESH, "non-manifold edge (" + std::to_string(ed[i].a) + ", " + std::to_string(ed[i].b) + ")"};
            return false;
        }
        nbr[ed[i].a].push_back(ed[i].b);
        nbr[ed[i].b].push_back(ed[i].a);
        if (cnt == 1) {
            T.bnd_vertex[ed[i].a] = T.bnd_vertex[ed[i].b] = 1;
        } else {
            const Ed &x = ed[i], &y = ed[i + 1];
            T.nb_face[x.f * 4 + x.k] = y.f;
            T.nb_edge[x.f * 4 + x.k] = y.k;
            T.nb_face[y.f * 4 + y.k] = x.f;
            T.nb_edge[y.f * 4 + y.k] = x.k;
        }
        i = j;
    }
    T.valence.assign(V, 0);
    for (int64_t v = 0; v < V; ++v) T.valence[v] = (int32_t)nbr[v].size();
    T.vf_ptr.assign(V + 1, 0);
    for (int64_t f = 0; f < F; ++f)
        for (int c = 0; c < 4; ++c) T.vf_ptr[T.quads[f * 4 + c] + 1]++;
    for (int64_t v = 0; v < V; ++v) T.vf_ptr[v + 1] += T.vf_ptr[v];
    T.vf_face.assign(4 * F, 0);
    T.vf_corner.assign(4 * F, 0);
    {
        std::vector<int64_t> fill(T.vf_ptr.begin(), T.vf_ptr.end() - 1);
        for (int64_t f = 0; f < F; ++f)
            for (int c = 0; c < 4; ++c) {
                int32_t v = T.quads[f * 4 + c];
                T.vf_face[fill[v]] = (int32_t)f;
                T.vf_corner[fill[v]] = (int8_t)c;
                fill[v]++;
            }
    }
    T.is_ep.assign(V, 0);
    for (int64_t v = 0; v < V; ++v) {
        bool used = T.vf_ptr[v + 1] > T.vf_ptr[v];
        if (!used) continue;
        T.is_ep[v] = (!T.bnd_vertex[v] && T.valence[v] != 4) || (T.bnd_vertex[v] && T.valence[v] > 3);
    }
    // classification (Sec. 3)
    T.passive.assign(F, 0);
    T.irregular.assign(F, 0);
    for (int64_t f = 0; f < F; ++f)
        for (int c = 0; c < 4; ++c) {
            int32_t v = T.quads[f * 4 + c];
            if (T.bnd_vertex[v]) T.passive[f] = 1;
            if (T.is_ep[v]) T.irregular[f] = 1;
        }
    std::vector<uint8_t> passive_vertex(V, 0);
    for (int64_t f = 0; f < F; ++f)
        if (T.passive[f])
            for (int c = 0; c < 4; ++c) {
                int32_t v = T.quads[f * 4 + c];
                passive_vertex[v] = 1;
                if (T.is_ep[v]) {
                    err = {WQ_ERR_MESH, "EP " + std::to_string(v) + " lies in the 1-ring neighbourhood of the boundary"};
                    return false;
                }
            }
    T.boundary.assign(F, 0);
    for (int64_t f = 0; f < F; ++f)
        if (!T.passive[f])
            for (int c = 0; c < 4; ++c)
                if (passive_vertex[T.quads[f * 4 + c]]) T.boundary[f] = 1;
    T.enriched.assign(F, 0);
    if (mesh.level0_face) {
        std::unordered_set<int32_t> irr;
        for (int64_t f = 0; f < F; ++f)
            if (T.irregular[f] && mesh.level0_face[f] >= 0) irr.insert(mesh.level0_face[f]);
        for (int64_t f = 0; f < F; ++f)
            T.enriched[f] = (mesh.level0_face[f] >= 0 && irr.count(mesh.level0_face[f])) || T.irregular[f];
    } else {
        for (int64_t f = 0; f < F; ++f) T.enriched[f] = T.irregular[f];
    }
    std::vector<uint8_t> tpt(V, 0);
    for (int64_t v = 0; v < V; ++v) {
        bool any_e = false, any_n = false;
        for (int64_t p = T.vf_ptr[v]; p < T.vf_ptr[v + 1]; ++p) {
            if (T.enriched[T.vf_face[p]]) any_e = true; else any_n = true;
        }
        tpt[v] = any_e && any_n;
    }
    T.transition.assign(F, 0);
    T.etype.assign(F, REGULAR);
    for (int64_t f = 0; f < F; ++f) {
        for (int c = 0; c < 4; ++c)
            if (tpt[T.quads[f * 4 + c]]) T.transition[f] = 1;
        int8_t t = REGULAR;
        if (T.passive[f]) t = PASSIVE;
        else if (T.boundary[f]) t = BOUNDARY;
        else if (T.irregular[f]) t = IRREGULAR;
        else if (T.enriched[f] && T.transition[f]) t = ENR_TRANSITION;
        else if (T.transition[f]) t = TRANSITION;
        else if (T.enriched[f]) t = ENR_REGULAR;
        T.etype[f] = t;
    }
    // knot spans: 0 on a pair of opposite edges if either edge has exactly one boundary end
    T.span.assign(2 * F, 1.0);
    for (int64_t f = 0; f < F; ++f)
        for (int d = 0; d < 2; ++d)
            for (int k = d; k < 4; k += 2) {
                int32_t a = T.quads[f * 4 + k], b = T.quads[f * 4 + (k + 1) % 4];
                if (T.bnd_vertex[a] != T.bnd_vertex[b]) T.span[f * 2 + d] = 0.0;
            }
    return true;
}

// ------------------------------------------------------ sparse combinations
struct Term { int64_t k; double v; };
using Lin = std::vector<Term>;

static void lin_normalize(Lin& a) {
    std::sort(a.begin(), a.end(), [](const Term& x, const Term& y) { return x.k < y.k; });
    size_t o = 0;
    for (size_t i = 0; i < a.size();) {
        Term t = a[i++];
        while (i < a.size() && a[i].k == t.k) t.v += a[i++].v;
        a[o++] = t;
    }
    a.resize(o);
}

struct LinBuilder {
    Lin acc;
    LinBuilder& add(double w, const Lin& a) {
        if (w != 0.0)
            for (const Term& t : a) acc.push_back({t.k, w * t.v});
        return *this;
    }
    Lin done() { lin_normalize(acc); return std::move(acc); }
};

static std::vector<Lin> split7(const Lin* b0, const Lin* b1, const Lin* b2, const Lin* b3) {
    std::vector<Lin> o(7);
    o[0] = *b0;
    o[1] = LinBuilder().add(0.5, *b0).add(0.5, *b1).done();
    o[2] = LinBuilder().add(0.25, *b0).add(0.5, *b1).add(0.25, *b2).done();
    o[3] = LinBuilder().add(0.125, *b0).add(0.375, *b1).add(0.375, *b2).add(0.125, *b3).done();
    o[4] = LinBuilder().add(0.25, *b1).add(0.5, *b2).add(0.25, *b3).done();
    o[5] = LinBuilder().add(0.5, *b2).add(0.5, *b3).done();
    o[6] = *b3;
    return o;
}

static inline void dmap(int c, int i, int j, int& x, int& y) {
    switch (c) {
        case 0: x = i; y = j; break;
        case 1: x = 6 - j; y = i; break;
        case 2: x = 6 - i; y = 6 - j; break;
        default: x = j; y = 6 - i; break;
    }
}

// B-spline inner Bezier point of face f next to corner c as weights of the face's
// four corner vertices: the legs are divided in the ratio of the knot spans on
// either side (Boehm's B-spline-to-Bezier rule).  False on degenerate spans.
static bool leg_division(const Topology& T, int64_t f, int c, double w[4]) {
    double du = T.span[f * 2], dv = T.span[f * 2 + 1];
    double dum = T.cross_span(f, 3), dup = T.cross_span(f, 1);
    double dvm = T.cross_span(f, 0), dvp = T.cross_span(f, 2);
    double su = dum + du + dup, sv = dvm + dv + dvp;
    if (!(su > 0) || !(sv > 0)) return false;
    double a = (dum + (CU[c] ? du : 0.0)) / su;
    double b = (dvm + (CV[c] ? dv : 0.0)) / sv;
    w[0] = (1 - a) * (1 - b);
    w[1] = a * (1 - b);
    w[2] = a * b;
    w[3] = (1 - a) * b;
    return true;
}

namespace {
struct NetBuilder {
    const Topology& T;
    std::vector<int64_t> erank;
    std::vector<Lin> inner_cache;   // [F][4]
    std::vector<uint8_t> have;

    NetBuilder(const Topology& t) : T(t) {
        erank.assign(T.F, -1);
        int64_t r = 0;
        for (int64_t f = 0; f < T.F; ++f)
            if (T.enriched[f]) erank[f] = r++;
        inner_cache.resize(4 * T.F);
        have.assign(4 * T.F, 0);
    }
    int64_t fdof(int64_t f, int c) const { return T.V + 4 * erank[f] + c; }

    const Lin& inner(int64_t f, int c, Error& err, bool& ok) {
        size_t key = f * 4 + c;
        if (have[key]) return inner_cache[key];
        Lin out;
        if (T.enriched[f]) {
            out.push_back({fdof(f, c), 1.0});
        } else {
            double w[4];
            if (!leg_division(T, f, c, w)) {
                err = {WQ_ERR_MESH, "degenerate knot spans around face " + std::to_string(f)};
                ok = false;
                return inner_cache[key];
            }
            for (int cc = 0; cc < 4; ++cc)
                if (w[cc] != 0.0) out.push_back({(int64_t)T.quads[f * 4 + cc], w[cc]});
            lin_normalize(out);
        }
        inner_cache[key] = std::move(out);
        have[key] = 1;
        return inner_cache[key];
    }

    Lin edge_point(int64_t f, int k, int c, Error& err, bool& ok) {
        int32_t g = T.nb_face[f * 4 + k];
        int kg = T.nb_edge[f * 4 + k];
        if (g < 0) {
            err = {WQ_ERR_MESH, "active face " + std::to_string(f) + " has a boundary edge"};
            ok = false;
            return Lin();
        }
        double df = T.span[f * 2 + ((k + 1) & 1)];
        double dg = T.span[g * 2 + ((kg + 1) & 1)];
        int32_t v = T.quads[f * 4 + c];
        const Lin& a = inner(f, c, err, ok);
        const Lin& b = inner(g, T.corner_of(g, v), err, ok);
        return LinBuilder().add(dg / (df + dg), a).add(df / (df + dg), b).done();
    }

    Lin corner_point(int64_t f, int c, Error& err, bool& ok) {
        int32_t v = T.quads[f * 4 + c];
        if (T.bnd_vertex[v]) {
            err = {WQ_ERR_MESH, "active face " + std::to_string(f) + " touches the boundary"};
            ok = false;
            return Lin();
        }
        int64_t p0 = T.vf_ptr[v], p1 = T.vf_ptr[v + 1];
        if (T.is_ep[v] || T.valence[v] != 4) {
            LinBuilder lb;
            double w = 1.0 / (double)(p1 - p0);
            for (int64_t p = p0; p < p1; ++p) lb.add(w, inner(T.vf_face[p], T.vf_corner[p], err, ok));
            return lb.done();
        }
        int ka = (c + 3) % 4, kb = c;
        int32_t ga = T.nb_face[f * 4 + ka], gb = T.nb_face[f * 4 + kb];
        int kga = T.nb_edge[f * 4 + ka], kgb = T.nb_edge[f * 4 + kb];
        int32_t d = -1;
        for (int64_t p = p0; p < p1; ++p) {
            int32_t h = T.vf_face[p];
            if (h != f && h != ga && h != gb) d = h;
        }
        if (ga < 0 || gb < 0 || d < 0) {
            err = {WQ_ERR_MESH, "vertex " + std::to_string(v) + " has a broken fan"};
            ok = false;
            return Lin();
        }
        double dxp = T.span[f * 2 + ((ka + 1) & 1)], dxm = T.span[ga * 2 + ((kga + 1) & 1)];
        double dyp = T.span[f * 2 + ((kb + 1) & 1)], dym = T.span[gb * 2 + ((kgb + 1) & 1)];
        double den = (dxm + dxp) * (dym + dyp);
        return LinBuilder()
            .add(dxm * dym / den, inner(f, c, err, ok))
            .add(dxp * dym / den, inner(ga, T.corner_of(ga, v), err, ok))
            .add(dxm * dyp / den, inner(gb, T.corner_of(gb, v), err, ok))
            .add(dxp * dyp / den, inner(d, T.corner_of(d, v), err, ok))
            .done();
    }

    // 4x4 net, index i*4 + j (i along corner0->corner1, j along corner0->corner3)
    bool net(int64_t f, std::vector<Lin>& b, Error& err) {
        bool ok = true;
        b.assign(16, Lin());
        auto at = [&](int i, int j) -> Lin& { return b[i * 4 + j]; };
        at(0, 0) = corner_point(f, 0, err, ok);
        at(3, 0) = corner_point(f, 1, err, ok);
        at(3, 3) = corner_point(f, 2, err, ok);
        at(0, 3) = corner_point(f, 3, err, ok);
        at(1, 1) = inner(f, 0, err, ok);
        at(2, 1) = inner(f, 1, err, ok);
        at(2, 2) = inner(f, 2, err, ok);
        at(1, 2) = inner(f, 3, err, ok);
        at(1, 0) = edge_point(f, 0, 0, err, ok);
        at(2, 0) = edge_point(f, 0, 1, err, ok);
        at(3, 1) = edge_point(f, 1, 1, err, ok);
        at(3, 2) = edge_point(f, 1, 2, err, ok);
        at(2, 3) = edge_point(f, 2, 2, err, ok);
        at(1, 3) = edge_point(f, 2, 3, err, ok);
        at(0, 2) = edge_point(f, 3, 3, err, ok);
        at(0, 1) = edge_point(f, 3, 0, err, ok);
        return ok;
    }
};
}  // namespace

// counter-clockwise fan (face, corner) around interior vertex v
bool fan(const Topology& T, int32_t v, std::vector<std::pair<int32_t, int>>& out, Error& err) {
    out.clear();
    int32_t f = T.vf_face[T.vf_ptr[v]];
    int c = T.vf_corner[T.vf_ptr[v]];
    out.push_back({f, c});
    for (int it = 0; it < 64; ++it) {
        int32_t g = T.nb_face[f * 4 + (c + 3) % 4];
        if (g < 0) {
            err = {WQ_ERR_MESH, "EP " + std::to_string(v) + " is not interior"};
            return false;
        }
        if (g == out[0].first) break;
        int cg = T.corner_of(g, v);
        out.push_back({g, cg});
        f = g;
        c = cg;
    }
    if ((int64_t)out.size() != T.vf_ptr[v + 1] - T.vf_ptr[v]) {
        err = {WQ_ERR_MESH, "EP " + std::to_string(v) + " has a non-manifold fan"};
        return false;
    }
    return true;
}

bool build_basis(const wq_mesh_desc& mesh, BasisHost& B, Error& err) {
    if (!build_topology(mesh, B.topo, err)) return false;
    const Topology& T = B.topo;
    B.dim = mesh.dim;
    B.V = T.V;
    B.xyz.assign(mesh.xyz, mesh.xyz + 3 * T.V);
    NetBuilder NB(T);
    const int64_t F = T.F;
    // nets of active faces; split irregular ones into 7x7
    std::vector<std::vector<Lin>> nets(F);
    std::vector<std::vector<Lin>> split(F);   // 49 entries, x*7 + y
    for (int64_t f = 0; f < F; ++f) {
        if (T.passive[f]) continue;
        if (!NB.net(f, nets[f], err)) return false;
        if (T.irregular[f]) {
            std::vector<std::vector<Lin>> rows(4);   // rows[j][x]
            for (int j = 0; j < 4; ++j)
                rows[j] = split7(&nets[f][0 * 4 + j], &nets[f][1 * 4 + j], &nets[f][2 * 4 + j], &nets[f][3 * 4 + j]);
            split[f].assign(49, Lin());
            for (int x = 0; x < 7; ++x) {
                std::vector<Lin> colv = split7(&rows[0][x], &rows[1][x], &rows[2][x], &rows[3][x]);
                for (int y = 0; y < 7; ++y) split[f][x * 7 + y] = std::move(colv[y]);
            }
        }
    }
    // D-patch treatment at every EP
    std::vector<std::pair<int32_t, int>> fn;
    for (int64_t v = 0; v < T.V; ++v) {
        if (!T.is_ep[v]) continue;
        if (!fan(T, (int32_t)v, fn, err)) return false;
        const int mu = (int)fn.size();
        int x, y;
        dmap(fn[0].second, 0, 0, x, y);
        Lin p = split[fn[0].first][x * 7 + y];
        std::vector<Lin> dt(mu);
        for (int k = 0; k < mu; ++k) {
            dmap(fn[k].second, 2, 0, x, y);
            dt[k] = LinBuilder().add(1.0, split[fn[k].first][x * 7 + y]).add(-1.0, p).done();
        }
        LinBuilder bx, by;
        for (int k = 0; k < mu; ++k) {
            double ang = 2.0 * M_PI * (double)k / (double)mu;
            bx.add(2.0 / mu * std::cos(ang), dt[k]);
            by.add(2.0 / mu * std::sin(ang), dt[k]);
        }
        Lin X = bx.done(), Y = by.done();
        std::vector<Lin> tn(mu);
        for (int k = 0; k < mu; ++k) {
            double ang = 2.0 * M_PI * (double)k / (double)mu;
            tn[k] = LinBuilder().add(1.0, p).add(std::cos(ang), X).add(std::sin(ang), Y).done();
        }
        for (int k = 0; k < mu; ++k) {
            std::vector<Lin>& C = split[fn[k].first];
            int c = fn[k].second;
            const Lin& t0 = tn[k];
            const Lin& t1 = tn[(k + 1) % mu];
            Lin mid = LinBuilder().add(0.5, t0).add(0.5, t1).done();
            dmap(c, 1, 0, x, y); C[x * 7 + y] = p;
            dmap(c, 0, 1, x, y); C[x * 7 + y] = p;
            dmap(c, 2, 0, x, y); C[x * 7 + y] = t0;
            dmap(c, 0, 2, x, y); C[x * 7 + y] = t1;
            dmap(c, 1, 1, x, y); C[x * 7 + y] = mid;
        }
    }
    // gather per active element
    std::vector<int32_t> elem_face;
    for (int64_t f = 0; f < F; ++f)
        if (!T.passive[f]) elem_face.push_back((int32_t)f);
    const int64_t E = (int64_t)elem_face.size();
    std::vector<std::vector<int64_t>> ekeys(E);
    std::vector<std::vector<double>> ecoef(E);
    std::vector<int32_t> nsub(E);
    for (int64_t e = 0; e < E; ++e) {
        int64_t f = elem_face[e];
        int ns = T.irregular[f] ? 4 : 1;
        nsub[e] = ns;
        // collect entry lists: position p = s*16 + i*4 + j
        std::vector<const Lin*> ent(ns * 16);
        for (int s = 0; s < ns; ++s)
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    if (ns == 1) ent[i * 4 + j] = &nets[f][i * 4 + j];
                    else {
                        int su = s & 1, sv = s >> 1;
                        ent[s * 16 + i * 4 + j] = &split[f][(3 * su + i) * 7 + (3 * sv + j)];
                    }
                }
        std::vector<int64_t> keys;
        for (const Lin* l : ent)
            for (const Term& t : *l) keys.push_back(t.k);
        std::sort(keys.begin(), keys.end());
        keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
        std::vector<double> co(keys.size() * ns * 16, 0.0);
        for (int p = 0; p < ns * 16; ++p)
            for (const Term& t : *ent[p]) {
                size_t idx = std::lower_bound(keys.begin(), keys.end(), t.k) - keys.begin();
                co[idx * ns * 16 + p] += t.v;
            }
        std::vector<int64_t> kk;
        std::vector<double> cc;
        for (size_t a = 0; a < keys.size(); ++a) {
            double mx = 0;
            for (int p = 0; p < ns * 16; ++p) mx = std::max(mx, std::fabs(co[a * ns * 16 + p]));
            if (mx > COEF_TOL) {
                kk.push_back(keys[a]);
                cc.insert(cc.end(), co.begin() + a * ns * 16, co.begin() + (a + 1) * ns * 16);
            }
        }
        ekeys[e] = std::move(kk);
        ecoef[e] = std::move(cc);
    }
    // numbering
    std::vector<int64_t> used;
    for (auto& k : ekeys) used.insert(used.end(), k.begin(), k.end());
    std::sort(used.begin(), used.end());
    used.erase(std::unique(used.begin(), used.end()), used.end());
    B.raw_ids = used;
    B.n = (int64_t)used.size();
    B.E = E;
    B.elem_face = elem_face;
    B.nsub = nsub;
    B.etype.resize(E);
    B.fn_ptr.assign(E + 1, 0);
    B.coef_ptr.assign(E + 1, 0);
    B.sub_ptr.assign(E + 1, 0);
    for (int64_t e = 0; e < E; ++e) {
        B.etype[e] = T.etype[elem_face[e]];
        B.fn_ptr[e + 1] = B.fn_ptr[e] + (int64_t)ekeys[e].size();
        B.coef_ptr[e + 1] = B.coef_ptr[e] + (int64_t)ecoef[e].size();
        B.sub_ptr[e + 1] = B.sub_ptr[e] + nsub[e];
    }
    B.fns.resize(B.fn_ptr[E]);
    B.coef.resize(B.coef_ptr[E]);
    for (int64_t e = 0; e < E; ++e) {
        for (size_t a = 0; a < ekeys[e].size(); ++a)
            B.fns[B.fn_ptr[e] + a] = (int32_t)(std::lower_bound(used.begin(), used.end(), ekeys[e][a]) - used.begin());
        std::copy(ecoef[e].begin(), ecoef[e].end(), B.coef.begin() + B.coef_ptr[e]);
    }
    // positions of the face-based control points: given, or the B-spline inner
    // Bezier points of their faces
    B.enr.clear();
    for (int64_t f = 0; f < F; ++f)
        if (T.enriched[f]) B.enr.push_back((int32_t)f);
    const size_t n_enr = B.enr.size();
    if (mesh.face_xyz) {
        if (mesh.n_face_xyz != (int64_t)(4 * n_enr)) {
            err = {WQ_ERR_ARG, "face_xyz holds " + std::to_string(mesh.n_face_xyz) + " points, the mesh has " +
                                   std::to_string(n_enr) + " enriched faces (4 points each)"};
            return false;
        }
        B.face_xyz.assign(mesh.face_xyz, mesh.face_xyz + 12 * n_enr);
    } else {
        B.face_xyz.assign(12 * n_enr, 0.0);
        for (size_t r = 0; r < n_enr; ++r) {
            const int64_t f = B.enr[r];
            const int32_t* q = &T.quads[f * 4];
            for (int c = 0; c < 4; ++c) {
                double w[4];
                if (!leg_division(T, f, c, w)) {
                    err = {WQ_ERR_MESH, "degenerate knot spans around face " + std::to_string(f)};
                    return false;
                }
                for (int cc = 0; cc < 4; ++cc)
                    for (int d = 0; d < 3; ++d) B.face_xyz[(4 * r + c) * 3 + d] += w[cc] * B.xyz[q[cc] * 3 + d];
            }
        }
    }
    B.level0.resize(F);
    for (int64_t f = 0; f < F; ++f) B.level0[f] = mesh.level0_face ? mesh.level0_face[f] : (int32_t)f;
    // control points of the functions
    B.ctrl.assign(3 * B.n, 0.0);
    for (int64_t i = 0; i < B.n; ++i) {
        int64_t k = used[i];
        const double* src = k < T.V ? &B.xyz[k * 3] : &B.face_xyz[(k - T.V) * 3];
        for (int d = 0; d < 3; ++d) B.ctrl[i * 3 + d] = src[d];
    }
    // geometry nets relative to the control point of the element's first function:
    // x = ref + sum_j c_j (P_j - ref) (partition of unity), so that derivatives of the
    // geometry do not cancel absolute coordinates
    B.geom.assign(48 * B.sub_ptr[E], 0.0);
    B.geom_ref.assign(3 * E, 0.0);
    for (int64_t e = 0; e < E; ++e) {
        int ns = nsub[e];
        int32_t m = B.m(e);
        double* G = &B.geom[48 * B.sub_ptr[e]];
        const double* C = &B.coef[B.coef_ptr[e]];
        const double* ref = &B.ctrl[3 * B.fns[B.fn_ptr[e]]];
        for (int d = 0; d < 3; ++d) B.geom_ref[3 * e + d] = ref[d];
        for (int32_t a = 0; a < m; ++a) {
            const double* P = &B.ctrl[3 * B.fns[B.fn_ptr[e] + a]];
            const double rel[3] = {P[0] - ref[0], P[1] - ref[1], P[2] - ref[2]};
            for (int p = 0; p < ns * 16; ++p) {
                double w = C[a * ns * 16 + p];
                for (int d = 0; d < 3; ++d) G[p * 3 + d] += w * rel[d];
            }
        }
    }
    // supports and pattern S_i (Eq. 10)
    B.supp_ptr.assign(B.n + 1, 0);
    for (int64_t p = 0; p < B.fn_ptr[E]; ++p) B.supp_ptr[B.fns[p] + 1]++;
    for (int64_t i = 0; i < B.n; ++i) B.supp_ptr[i + 1] += B.supp_ptr[i];
    B.supp.resize(B.supp_ptr[B.n]);
    {
        std::vector<int64_t> fill(B.supp_ptr.begin(), B.supp_ptr.end() - 1);
        for (int64_t e = 0; e < E; ++e)
            for (int64_t p = B.fn_ptr[e]; p < B.fn_ptr[e + 1]; ++p) B.supp[fill[B.fns[p]]++] = (int32_t)e;
    }
    B.row_ptr.assign(B.n + 1, 0);
    B.col.clear();
    std::vector<int32_t> mark(B.n, -1), tmp;
    for (int64_t i = 0; i < B.n; ++i) {
        tmp.clear();
        for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) {
            int32_t e = B.supp[s];
            for (int64_t p = B.fn_ptr[e]; p < B.fn_ptr[e + 1]; ++p) {
                int32_t j = B.fns[p];
                if (mark[j] != (int32_t)i) { mark[j] = (int32_t)i; tmp.push_back(j); }
            }
        }
        std::sort(tmp.begin(), tmp.end());
        B.col.insert(B.col.end(), tmp.begin(), tmp.end());
        B.row_ptr[i + 1] = (int64_t)B.col.size();
        B.max_n_i = std::max<int32_t>(B.max_n_i, (int32_t)tmp.size());
    }
    B.max_m = 0;
    B.n_irregular = 0;
    for (int64_t e = 0; e < E; ++e) {
        B.max_m = std::max(B.max_m, B.m(e));
        B.n_irregular += (nsub[e] == 4);
    }
    for (int k = 0; k < 7; ++k) B.type_count[k] = 0;
    for (int64_t f = 0; f < F; ++f) B.type_count[T.etype[f]]++;
    return true;
}

// ---------------------------------------------- min-max counts (Sec. 4.2)
// Table 2's fixed sides; non-enriched transition and enriched regular elements get
// 4 x 4 when two or more EPs, or one of valence >= 7, lie among the vertices of the
// union of the supports of the functions active on the element, else 3 x 3.
static void table2_sides(const BasisHost& B, std::vector<int32_t>& side) {
    const Topology& T = B.topo;
    side.assign(B.E, 2);
    std::vector<int64_t> mark_e(B.E, -1), mark_v(T.V, -1);
    for (int64_t e = 0; e < B.E; ++e) {
        switch (B.etype[e]) {
            case REGULAR: side[e] = 2; continue;
            case BOUNDARY: case IRREGULAR: case ENR_TRANSITION: side[e] = 4; continue;
            default: break;
        }
        int n_ep = 0;
        bool high = false;
        for (int64_t p = B.fn_ptr[e]; p < B.fn_ptr[e + 1]; ++p) {
            const int32_t i = B.fns[p];
            for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) {
                const int32_t k = B.supp[s];
                if (mark_e[k] == e) continue;
                mark_e[k] = e;
                const int32_t f = B.elem_face[k];
                for (int c = 0; c < 4; ++c) {
                    const int32_t v = T.quads[(int64_t)f * 4 + c];
                    if (mark_v[v] == e) continue;
                    mark_v[v] = e;
                    if (T.is_ep[v]) {
                        ++n_ep;
                        high = high || T.valence[v] >= 7;
                    }
                }
            }
        }
        side[e] = (n_ep >= 2 || high) ? 4 : 3;
    }
}

bool point_counts(const BasisHost& B, int mode, std::vector<int32_t>& side, Error& err) {
    if (mode != WQ_COUNT_MINMAX && mode != WQ_COUNT_TABLE2) {
        err = {WQ_ERR_ARG, "unknown count mode"};
        return false;
    }
    const int64_t E = B.E;
    std::vector<uint8_t> isR(E);
    for (int64_t e = 0; e < E; ++e) isR[e] = (B.etype[e] == REGULAR || B.etype[e] == BOUNDARY);
    if (mode == WQ_COUNT_TABLE2) {
        table2_sides(B, side);
        return repair_counts(B, isR, side, err);
    }
    side.assign(E, 2);
    for (int64_t e = 0; e < E; ++e)
        if (B.etype[e] == BOUNDARY) side[e] = 4;
    for (int64_t i = 0; i < B.n; ++i) {
        int64_t n_i = B.row_ptr[i + 1] - B.row_ptr[i];
        int64_t er = 0, eb = 0, den = 0;
        bool any = false;
        for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) {
            int32_t k = B.supp[s];
            if (B.etype[k] == REGULAR) er++;
            else if (B.etype[k] == BOUNDARY) eb++;
            else { den += B.m(k); any = true; }
        }
        if (!any) continue;
        int64_t num = n_i - 4 * er - 16 * eb;
        if (num <= 0) continue;
        for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) {
            int32_t k = B.supp[s];
            if (isR[k]) continue;
            int64_t sk = 2;
            while (sk * sk * den < (int64_t)B.m(k) * num) ++sk;
            side[k] = std::max<int32_t>(side[k], (int32_t)sk);
        }
    }
    return repair_counts(B, isR, side, err);
}

// Raise the non-regular element with most functions (lowest id on ties) of every
// test function with fewer points than n_i until all are well posed (Sec. 4.2).
bool repair_counts(const BasisHost& B, const std::vector<uint8_t>& isR, std::vector<int32_t>& side, Error& err) {
    bool changed = true;
    while (changed) {
        changed = false;
        for (int64_t i = 0; i < B.n; ++i) {
            int64_t n_i = B.row_ptr[i + 1] - B.row_ptr[i], tot = 0;
            for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) tot += (int64_t)side[B.supp[s]] * side[B.supp[s]];
            if (tot >= n_i) continue;
            int32_t best = -1;
            for (int64_t s = B.supp_ptr[i]; s < B.supp_ptr[i + 1]; ++s) {
                int32_t k = B.supp[s];
                if (isR[k]) continue;
                if (best < 0 || B.m(k) > B.m(best) || (B.m(k) == B.m(best) && k < best)) best = k;
            }
            if (best < 0) {
                err = {WQ_ERR_ILLPOSED, "test function " + std::to_string(i) + " cannot be made well-posed"};
                return false;
            }
            side[best]++;
            changed = true;
        }
    }
    return true;
}

}  // namespace wqi
