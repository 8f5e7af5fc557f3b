// Host plan of one global refinement of a bicubic ASUTS control mesh (Sec. 3):
// the enriched region keeps its size, vertex-based control points come from knot
// insertion, face-based ones from de Casteljau's algorithm.
//
// Topology: a face is halved in every direction whose knot span is non-zero
// (active faces 2 x 2, faces of the passive ring 1 x 2 along the boundary, the
// passive corner faces whole).  Fine vertices: the coarse vertices [0, V), one
// per split edge in the order edges are first met scanning faces f = 0..F-1 and
// their edges k = 0..3, one per 2 x 2-split face centre in face order.  Fine faces
// in coarse face order; children of a 2 x 2 split by the coarse corner they
// contain, of a 1 x 2 split by increasing coordinate; every child keeps its
// parent's orientation and initial-mesh face.
//
// Vertex-based points: in the tensor chart of the fine vertex's parent (coarse
// vertex, edge or face) the midpoints of the non-zero knot spans are inserted in
// each direction; the fine point is the tensor product of the one-dimensional
// rules below.  They are Boehm's insertion written out with blossoms: a cubic
// control point d_j = f(t_{j-1}, t_j, t_{j+1}) belongs to knot t_j, and the fine
// points are f(m_{j-1}, t_j, m_j) (at t_j) and f(t_j, m_j, t_{j+1}) (at the
// midpoint m_j).  Spans beyond the chart are the cross spans of the neighbouring
// faces (0 beyond the boundary).  Vertices of the outer boundary loop have zero
// spans on both sides across the boundary: only the rule along the loop acts.
// At an EP (no tensor chart) the fine point keeps the coarse position; the EP
// function is eliminated at every level, so this value enters no function.
//
// Face-based points: for every coarse enriched face, the element's Bezier
// coefficients and function ids; the device contracts them with the coarse
// control points into the face's net, splits it at 1/2 (de Casteljau) and
// writes the inner points of the four children (k_refine.cu).
#include <algorithm>
#include <array>
#include <map>
#include <string>
#include <utility>

#include "wq_internal.h"

namespace wqi {

// Fine control point at t_0 as weights of (d_{-1}, d_0, d_1); spans D_j = t_{j+1} - t_j.
static void rule_vertex(double Dm2, double Dm1, double D0, double D1, double w[3]) {
    if (!(Dm1 + D0 > 0.0)) {
        w[0] = 0.0, w[1] = 1.0, w[2] = 0.0;
        return;
    }
    // E = f(t_0, t_1, m_0) = d_0 + lam (d_1 - d_0)
    const double lam = (Dm1 + 0.5 * D0) / (Dm1 + D0 + D1);
    // L = f(t_-1, t_0, m_0) = d_-1 + kap (d_0 - d_-1)
    const double kap = (Dm2 + Dm1 + 0.5 * D0) / (Dm2 + Dm1 + D0);
    // f(m_-1, t_0, m_0) = L + rho (E - L)
    const double rho = 0.5 * Dm1 / (Dm1 + D0);
    w[0] = (1.0 - rho) * (1.0 - kap);
    w[1] = (1.0 - rho) * kap + rho * (1.0 - lam);
    w[2] = rho * lam;
}

// Fine control point at the midpoint of D_0 > 0: weight of d_1 (d_0 takes 1 - lam).
static double rule_edge(double Dm1, double D0, double D1) { return (Dm1 + 0.5 * D0) / (Dm1 + D0 + D1); }

static inline int64_t ekey(int32_t a, int32_t b) {
    return a < b ? ((int64_t)a << 32) | (uint32_t)b : ((int64_t)b << 32) | (uint32_t)a;
}

bool build_refine(const BasisHost& B, RefinePlan& R, Error& err) {
    const Topology& T = B.topo;
    const int64_t V = T.V, F = T.F;
    const int32_t* q = T.quads.data();
    auto span = [&](int64_t f, int a) { return T.span[f * 2 + a]; };
    auto qv = [&](int64_t f, int c) { return q[f * 4 + (c & 3)]; };

    // ---------------------------------------------------------------- edges
    std::map<int64_t, std::pair<double, int>> edges;   // key -> (span, faces)
    for (int64_t f = 0; f < F; ++f)
        for (int k = 0; k < 4; ++k) {
            const int64_t key = ekey(qv(f, k), qv(f, k + 1));
            const double sp = span(f, k & 1);
            auto it = edges.find(key);
            if (it == edges.end()) {
                edges[key] = {sp, 1};
            } else {
                if ((it->second.first > 0) != (sp > 0)) {
                    err = {WQ_ERR_MESH, "edge of face " + std::to_string(f) + " has inconsistent knot spans"};
                    return false;
                }
                it->second.second += 1;
            }
        }
    auto span_of = [&](int32_t a, int32_t b) { return edges.at(ekey(a, b)).first; };

    // ------------------------------------------------------------- topology
    std::map<int64_t, int32_t> mid;
    std::vector<std::pair<int64_t, int>> edge_parent;
    int64_t nv = V;
    for (int64_t f = 0; f < F; ++f)
        for (int k = 0; k < 4; ++k) {
            const int64_t key = ekey(qv(f, k), qv(f, k + 1));
            if (edges[key].first > 0 && !mid.count(key)) {
                mid[key] = (int32_t)nv++;
                edge_parent.push_back({f, k});
            }
        }
    std::vector<int32_t> centre(F, -1);
    for (int64_t f = 0; f < F; ++f)
        if (span(f, 0) > 0 && span(f, 1) > 0) centre[f] = (int32_t)nv++;
    if (nv > INT32_MAX) {
        err = {WQ_ERR_ARG, "refined mesh too large for 32-bit indices"};
        return false;
    }
    auto m = [&](int64_t f, int k) { return mid.at(ekey(qv(f, k), qv(f, k + 1))); };
    R.quads.clear();
    R.level0.clear();
    for (int64_t f = 0; f < F; ++f) {
        const int32_t c0 = qv(f, 0), c1 = qv(f, 1), c2 = qv(f, 2), c3 = qv(f, 3);
        const bool su = span(f, 0) > 0, sv = span(f, 1) > 0;
        std::vector<std::array<int32_t, 4>> kids;
        if (su && sv) {
            const int32_t z = centre[f];
            kids = {{c0, m(f, 0), z, m(f, 3)}, {m(f, 0), c1, m(f, 1), z}, {z, m(f, 1), c2, m(f, 2)},
                    {m(f, 3), z, m(f, 2), c3}};
        } else if (su) {
            kids = {{c0, m(f, 0), m(f, 2), c3}, {m(f, 0), c1, c2, m(f, 2)}};
        } else if (sv) {
            kids = {{c0, c1, m(f, 1), m(f, 3)}, {m(f, 3), m(f, 1), c2, c3}};
        } else {
            kids = {{c0, c1, c2, c3}};
        }
        for (auto& kq : kids) {
            R.quads.insert(R.quads.end(), kq.begin(), kq.end());
            R.level0.push_back(B.level0[f]);
        }
    }
    R.Vc = V;
    R.Vf = nv;
    R.Ff = (int64_t)R.level0.size();

    // ------------------------------------------------- vertex-based points
    R.st_ptr.assign(nv + 1, 0);
    std::vector<std::vector<std::pair<int32_t, double>>> st(nv);
    // boundary loop neighbours: edges of exactly one face
    std::vector<std::vector<int32_t>> bloop(V);
    for (auto& e : edges)
        if (e.second.second == 1) {
            const int32_t a = (int32_t)(e.first >> 32), b = (int32_t)(e.first & 0xffffffff);
            bloop[a].push_back(b);
            bloop[b].push_back(a);
        }
    std::vector<std::pair<int32_t, int>> fn;
    for (int64_t v = 0; v < V; ++v) {
        if (T.vf_ptr[v + 1] == T.vf_ptr[v] || T.is_ep[v]) {
            st[v] = {{(int32_t)v, 1.0}};
            continue;
        }
        if (T.bnd_vertex[v]) {
            if (bloop[v].size() != 2) {
                err = {WQ_ERR_MESH, "boundary vertex " + std::to_string(v) + " has " +
                                        std::to_string(bloop[v].size()) + " boundary edges"};
                return false;
            }
            const int32_t p = bloop[v][0], n = bloop[v][1];
            if (bloop[p].size() != 2 || bloop[n].size() != 2) {
                err = {WQ_ERR_MESH, "boundary loop is not a simple cycle near vertex " + std::to_string(v)};
                return false;
            }
            const int32_t pp = bloop[p][0] == (int32_t)v ? bloop[p][1] : bloop[p][0];
            const int32_t nn = bloop[n][0] == (int32_t)v ? bloop[n][1] : bloop[n][0];
            double w[3];
            rule_vertex(span_of(pp, p), span_of(p, (int32_t)v), span_of((int32_t)v, n), span_of(n, nn), w);
            const int32_t src[3] = {p, (int32_t)v, n};
            for (int i = 0; i < 3; ++i)
                if (w[i] != 0.0) st[v].push_back({src[i], w[i]});
            continue;
        }
        if (!fan(T, (int32_t)v, fn, err)) return false;
        if (fn.size() != 4) {
            err = {WQ_ERR_MESH, "interior vertex " + std::to_string(v) + " of valence " +
                                    std::to_string(fn.size()) + " is not marked extraordinary"};
            return false;
        }
        int32_t nb[4], dg[4];
        double beyond[4], sp[4];
        for (int k = 0; k < 4; ++k) {
            const int32_t f = fn[k].first;
            const int c = fn[k].second;
            nb[k] = qv(f, c + 1);
            dg[k] = qv(f, c + 2);
            beyond[k] = T.cross_span(f, (c + 1) & 3);
        }
        for (int k = 0; k < 4; ++k) sp[k] = span_of((int32_t)v, nb[k]);
        double a[3], b[3];
        rule_vertex(beyond[2], sp[2], sp[0], beyond[0], a);   // line n2 - v - n0
        rule_vertex(beyond[3], sp[3], sp[1], beyond[1], b);   // line n3 - v - n1
        // grid (i, j), i along n2 -> n0, j along n3 -> n1
        const int32_t grid[3][3] = {{dg[2], nb[2], dg[1]}, {nb[3], (int32_t)v, nb[1]}, {dg[3], nb[0], dg[0]}};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                const double w = a[i] * b[j];
                if (w != 0.0) st[v].push_back({grid[i][j], w});
            }
    }
    for (auto& ep : edge_parent) {
        const int64_t f = ep.first;
        const int k = ep.second;
        const int32_t a = qv(f, k), b = qv(f, k + 1);
        const int32_t w_id = m(f, k);
        const double lam = rule_edge(T.cross_span(f, (k + 3) & 3), span(f, k & 1), T.cross_span(f, (k + 1) & 3));
        // rows across the edge: -1 in the neighbour g, 0 the edge, +1 in f
        int32_t rows[3][2] = {{-1, -1}, {a, b}, {qv(f, k + 3), qv(f, k + 2)}};
        const int32_t g = T.nb_face[f * 4 + k];
        double across_g = 0.0, beyond_g = 0.0;
        if (g >= 0) {
            const int kg = T.nb_edge[f * 4 + k];
            rows[0][0] = qv(g, kg + 2);
            rows[0][1] = qv(g, kg + 3);
            across_g = span(g, (kg + 1) & 1);
            beyond_g = T.cross_span(g, (kg + 2) & 3);
        }
        double beta[3];
        rule_vertex(beyond_g, across_g, span(f, (k + 1) & 1), T.cross_span(f, (k + 2) & 3), beta);
        for (int r = 0; r < 3; ++r) {
            if (beta[r] == 0.0) continue;
            if (rows[r][0] < 0) {
                err = {WQ_ERR_MESH, "knot insertion at an edge of face " + std::to_string(f) + " needs a missing face"};
                return false;
            }
            st[w_id].push_back({rows[r][0], beta[r] * (1.0 - lam)});
            st[w_id].push_back({rows[r][1], beta[r] * lam});
        }
    }
    for (int64_t f = 0; f < F; ++f) {
        if (centre[f] < 0) continue;
        const double lu = rule_edge(T.cross_span(f, 3), span(f, 0), T.cross_span(f, 1));
        const double lv = rule_edge(T.cross_span(f, 0), span(f, 1), T.cross_span(f, 2));
        const double w[4] = {(1 - lu) * (1 - lv), lu * (1 - lv), lu * lv, (1 - lu) * lv};
        for (int c = 0; c < 4; ++c)
            if (w[c] != 0.0) st[centre[f]].push_back({qv(f, c), w[c]});
    }
    R.st_src.clear();
    R.st_w.clear();
    for (int64_t w = 0; w < nv; ++w) {
        R.st_ptr[w] = (int64_t)R.st_src.size();
        for (auto& e : st[w]) {
            R.st_src.push_back(e.first);
            R.st_w.push_back(e.second);
        }
    }
    R.st_ptr[nv] = (int64_t)R.st_src.size();

    // ------------------------------------------------- face-based points
    std::vector<int64_t> elem_of(F, -1);
    for (int64_t e = 0; e < B.E; ++e) elem_of[B.elem_face[e]] = e;
    R.jobs.clear();
    R.fn_raw.clear();
    R.coef.clear();
    R.n_fx_c = 4 * (int64_t)B.enr.size();
    for (size_t r = 0; r < B.enr.size(); ++r) {
        const int64_t f = B.enr[r];
        const int64_t e = elem_of[f];
        if (e < 0 || centre[f] < 0) {
            err = {WQ_ERR_MESH, "enriched face " + std::to_string(f) + " is not an active 2 x 2-split face"};
            return false;
        }
        RefineJob j;
        j.coef_off = (int64_t)R.coef.size();
        j.fn_off = (int32_t)R.fn_raw.size();
        j.m = B.m(e);
        j.nsub = B.nsub[e];
        j.out = (int32_t)(16 * r);
        for (int64_t p = B.fn_ptr[e]; p < B.fn_ptr[e + 1]; ++p) R.fn_raw.push_back((int32_t)B.raw_ids[B.fns[p]]);
        R.coef.insert(R.coef.end(), B.coef.begin() + B.coef_ptr[e], B.coef.begin() + B.coef_ptr[e + 1]);
        R.jobs.push_back(j);
    }
    if (R.fn_raw.size() > (size_t)INT32_MAX || R.n_fx_c > INT32_MAX / 4) {
        err = {WQ_ERR_ARG, "enriched region too large for 32-bit job offsets"};
        return false;
    }
    R.n_fx_f = 16 * (int64_t)B.enr.size();
    return true;
}

}  // namespace wqi
