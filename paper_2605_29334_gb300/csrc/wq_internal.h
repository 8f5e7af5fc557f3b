// Internal data structures of the WQ library (host side).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/wq.h"

namespace wqi {

enum ElemType { PASSIVE = 0, BOUNDARY = 1, IRREGULAR = 2, ENR_TRANSITION = 3, TRANSITION = 4,
                ENR_REGULAR = 5, REGULAR = 6 };

struct Error {
    wq_status code;
    std::string msg;
};

// Mesh topology and the classification of Sec. 3.
struct Topology {
    int64_t V = 0, F = 0;
    std::vector<int32_t> quads;          // [F][4]
    std::vector<int32_t> nb_face;        // [F][4] face across edge k (-1 none)
    std::vector<int8_t> nb_edge;         // [F][4] its local edge index
    std::vector<int64_t> vf_ptr;         // vertex -> incident (face, corner)
    std::vector<int32_t> vf_face;
    std::vector<int8_t> vf_corner;
    std::vector<uint8_t> bnd_vertex, is_ep;
    std::vector<int32_t> valence;
    std::vector<uint8_t> passive, boundary, irregular, enriched, transition;
    std::vector<int8_t> etype;           // per face
    std::vector<double> span;            // [F][2]

    double cross_span(int64_t f, int k) const {
        int32_t g = nb_face[f * 4 + k];
        if (g < 0) return 0.0;
        int kg = nb_edge[f * 4 + k];
        return span[g * 2 + ((kg + 1) & 1)];
    }
    int corner_of(int64_t f, int32_t v) const {
        for (int c = 0; c < 4; ++c)
            if (quads[f * 4 + c] == v) return c;
        return -1;
    }
};

// The spline space, element by element (active elements only).
struct BasisHost {
    int dim = 2;
    int64_t n = 0, E = 0, V = 0;
    Topology topo;
    std::vector<double> xyz;            // [V][3]
    std::vector<int32_t> level0;        // [F] initial-mesh face of every face (the face itself if none given)
    std::vector<int32_t> enr;           // enriched faces, ascending
    std::vector<double> face_xyz;       // [enr.size()][4][3] face-based control points
    std::vector<int32_t> elem_face;     // [E]
    std::vector<int8_t> etype;          // [E]
    std::vector<int32_t> nsub;          // [E] 1 or 4
    std::vector<int64_t> fn_ptr;        // [E+1]
    std::vector<int32_t> fns;           // function ids per element, ascending
    std::vector<int64_t> coef_ptr;      // [E+1] offsets into coef
    std::vector<double> coef;           // per element [m][nsub][4][4]
    std::vector<double> geom;           // per element [nsub][4][4][3] relative to geom_ref, offsets 48*sub_ptr
    std::vector<double> geom_ref;       // [E][3] control point of the element's first function
    std::vector<int64_t> sub_ptr;       // [E+1] prefix sums of nsub
    std::vector<double> ctrl;           // [n][3]
    std::vector<int64_t> raw_ids;       // [n]
    std::vector<int64_t> supp_ptr;      // [n+1]
    std::vector<int32_t> supp;          // ascending element ids
    std::vector<int64_t> row_ptr;       // [n+1] pattern of S_i
    std::vector<int32_t> col;           // sorted
    int32_t max_m = 0, max_n_i = 0;
    int64_t n_irregular = 0;
    int64_t type_count[7] = {0, 0, 0, 0, 0, 0, 0};

    int32_t m(int64_t e) const { return (int32_t)(fn_ptr[e + 1] - fn_ptr[e]); }
};

// One global refinement (Sec. 3): fine topology, knot-insertion stencils of the
// vertex-based control points, and the coarse enriched elements whose Bezier nets
// give the face-based control points (refine_host.cpp).
struct RefineJob {
    int64_t coef_off;     // element coefficients [m][nsub][4][4] in RefinePlan::coef
    int32_t fn_off;       // raw control-variable ids of its m functions in RefinePlan::fn_raw
    int32_t m, nsub;
    int32_t out;          // first fine face-based point written (16 per job)
};
struct RefinePlan {
    int64_t Vc = 0, n_fx_c = 0;           // coarse vertices, coarse face-based points
    int64_t Vf = 0, Ff = 0, n_fx_f = 0;   // fine vertices, faces, face-based points
    std::vector<int32_t> quads, level0;   // fine faces [Ff][4], [Ff]
    std::vector<int64_t> st_ptr;          // [Vf+1] stencil of every fine vertex
    std::vector<int32_t> st_src;          // coarse vertex ids
    std::vector<double> st_w;
    std::vector<RefineJob> jobs;          // one per coarse enriched face, ascending
    std::vector<int32_t> fn_raw;
    std::vector<double> coef;
};

// Host steps (host.cpp).  Return false and fill err on failure.
bool fan(const Topology& T, int32_t v, std::vector<std::pair<int32_t, int>>& out, Error& err);
bool build_refine(const BasisHost& B, RefinePlan& R, Error& err);
bool build_topology(const wq_mesh_desc& mesh, Topology& T, Error& err);
bool build_basis(const wq_mesh_desc& mesh, BasisHost& B, Error& err);
bool point_counts(const BasisHost& B, int mode, std::vector<int32_t>& side, Error& err);
bool repair_counts(const BasisHost& B, const std::vector<uint8_t>& isR, std::vector<int32_t>& side, Error& err);

}  // namespace wqi
