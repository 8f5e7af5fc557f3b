// Device-side views shared by the WQ kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wqd {

constexpr int WQ_TERMS_MAX = 8;   // terms of an operator (padded to 1, 2, 3, 4 or 8)

// Status flags written by kernels (bitwise OR into a device word).
enum : unsigned int {
    ST_NOT_CONVERGED = 1u,
    ST_NONFINITE = 2u,
    ST_ILLPOSED = 4u,
    ST_BAD_INDEX = 8u,
    ST_GEOMETRY = 16u,
    ST_TIMEOUT = 32u         // a bounded wait for staged data ran out (k_tile.cu)
};

// Per-element spline data and point tables of one rule.
struct Elems {
    int dim;                 // 2 or 3
    int nc;                  // table components: N, d_x, d_y, (d_z), lap  (= dim + 2)
    int64_t E;
    const int32_t* m;        // [E] functions on the element
    const int32_t* nsub;     // [E] 1 or 4
    const int32_t* side;     // [E] WQ grid side
    const int64_t* coef_ptr; // [E+1] into coef ([m][nsub][4][4])
    const double* coef;
    const int64_t* sub_ptr;  // [E+1]; geometry net of sub s of e at geom + 48*(sub_ptr[e]+s)
    const double* geom;      // [nsub][4][4][3] relative to geom_ref[e]
    const double* geom_ref;  // [E][3]
    const int64_t* pt_ptr;   // [E+1] WQ points of e
    const int64_t* gp_ptr;   // [E+1] Gauss points of e (16 nsub)
    const int64_t* bt_ptr;   // [E+1] WQ table of e: [P_e][nc][m_e]
    const int64_t* gbt_ptr;  // [E+1] Gauss table of e: [16 nsub][nc][m_e]
};

// Row (test function) plan: support elements and local positions.
struct Rows {
    int64_t n;
    const int32_t* row_ptr;   // [n+1] CSR pattern of S_i
    const int64_t* supp_ptr;  // [n+1]
    const int32_t* supp;      // support elements, ascending
    const int64_t* pos_ptr;   // [#supp + 1] into pos
    const uint16_t* pos;      // for support entry s (element e): position in row i of each local function of e
    const uint8_t* il;        // [#supp] local index of function i in element supp[s]
    const int64_t* w_ptr;     // [n+1] weights of row i at [w_ptr[i], w_ptr[i+1])
    const int32_t* order;     // [n] processing order of the rows (spatially sorted), or null
};

// One weight component of one rule for the batched truncated-SVD launch: the rule's
// element and row plans, its point table (component tc gives A, component 0 gives Z),
// moments [nnz], weights W (column wc of nwc), per-row rank / Z = I flags and status.
struct TsvdSet {
    Elems el;
    Rows rw;
    const double* table;
    int tc;
    const double* mom;
    double* W;
    int nwc, wc;
    int32_t* rank;
    uint8_t* zid;
    unsigned* status;
};

// Element-major FP32 assembly.  Work items are 16 x 16 tiles of element blocks:
// item[k] = {table offset, first point, m | P << 8 | (a0/16) << 16 | (b0/16) << 20,
// first row of the element in the element-major weights}, kb[k] = start of the
// element's m x m entries in scat.  scat[.] = kscr slot of a block entry;
// gptr[n] .. gptr[n+1] = the slots of CSR entry n (shared by the WQ and Gauss items,
// whose blocks have the same shape).
struct ElemItems {
    int64_t n;
    const int4* item;
    const int32_t* kb;
};
struct ElemPlan {
    const int32_t* scat;
    const int32_t* gptr;
    float2* kscr;
};

// One rule's data for the FP32 element-major kernels.
struct ElemSrc {
    ElemPlan ep;
    const float2* table2;   // split basis table at the item's points (WQ or Gauss)
    const float2* W2e;      // element-major split weights (WQ items)
    const double* gw;       // Gauss weights (Gauss items)
    int64_t nnz;
    int nc, nwc;
};

// One rule's data for the FP64 element-major kernels (the slot buffer holds doubles).
struct ElemSrc64 {
    const int32_t* scat;
    const int32_t* gptr;
    double* kscr;
    const double* table;    // basis table at the item's points (WQ or Gauss)
    const double* We;       // element-major FP64 weights (WQ items)
    const double* gw;       // Gauss weights (Gauss items)
    int64_t nnz;
    int nc, nwc;
};

// Tensor-core element contraction (WQ_PREC_TC).  Per tile, it2[k] = {first function
// of the element in the per-function arrays, offset of the element's trial-side slices
// in bs (words), element, P rounded up to 4}.  The trial side of element e (table
// component c, column block cb of 16 functions, quarter-chunk qq of 4 points) is stored
// in mma fragment order: per slice l, 2 x 8 x 2 words, word (p, g, nt) holding slice l
// of T[q][n] for q = 4 qq + 2 p (low half) and q + 1 (high half), column
// n = 16 cb + 8 nt + g, as bf16 integers of T 2^(8 - f_ec) (f_ec = fexp[e nc + c],
// 2^f_ec > max |T| over the element); lane (g, t4) of a half-chunk reads p = t4 % 2 of
// the quarter its t4 / 2 selects.  vmax[(fn + a) nv + v] bounds the test-side
// values of local function a over the element's points (v: weight column, or
// table component for Gauss items).
struct TcItems {
    int64_t n;
    const int4* item;
    const int32_t* kb;
    const int4* it2;
    int n_sm;               // multiprocessors (persistent grid size)
};
struct TcSrc {
    const int32_t* scat;
    float2* kscr;
    const int32_t* gptr;
    const float2* vsrc;     // test side: element-major split weights (WQ) or split table (Gauss)
    const float2* gw2;      // split Gauss weights (Gauss items)
    const uint32_t* bs;     // trial-side slices
    const int32_t* fexp;    // [E][nc]
    const float* vmax;      // [sum_e m_e][nv]
    int64_t nnz;
    int nc, nwc;
};
// Set-up of the trial-side slices: el[e] = {table offset, points, element-major weight
// row (WQ), first function}; bs_ptr[e] = the element's slice offset (words).
struct TcPrep {
    const int4* el;
    const int64_t* bs_ptr;
    uint32_t* bs;
    int32_t* fexp;
    float* vmax;
};

// Tile kernels (k_tile.cu).  Per rule and quadrature: element-major packs of the test
// side (S0: WQ weights, or Gauss weight x test table) and the trial side (T0: basis
// table), [16-function block][component][point][16] per element, zero beyond m_e.
struct TileSrc {
    const float2* S0;
    const float2* T0;
    float2* kslot;           // row-major slots (see RowSrc)
    const int32_t* kdst;     // [sum_e m_e]: slot block of element e's row a at kdst[fn_ptr[e] + a]
    const float* tmx;        // bounds of |T_hi| per (element, 16-function block, trial component)
    int n_test, n_trial;     // components of the test and trial packs
};
// item[k] = {test pack base, trial pack base (float2 units), first point of the element
// (coefficient rows), fn_ptr[e] (kdst)}; meta[k] = {m | P << 8 | (a0 / 16) << 16 | (b0 / 16) << 20 |
// ncb << 24, rule (batched launches), offset of the element in tmx, 0}.
struct TileJob {
    int64_t n_items;
    const int4* item;
    const int4* meta;
    TileSrc one;
    const TileSrc* srcs;     // per rule (batched launches, device array)
    unsigned* status;        // ST_TIMEOUT
};
// Terms of an operator for the tile kernels: staged component indices (test side from
// s_lo, s_n components; trial side from r_lo, r_n), coefficient row (-1: the constant
// (shi, slo)), rows cstride apart.
struct TileTerms {
    int nt;
    int tcomp[WQ_TERMS_MAX], rcomp[WQ_TERMS_MAX], crow[WQ_TERMS_MAX];
    float shi[WQ_TERMS_MAX], slo[WQ_TERMS_MAX];
    int ncrow;
    int64_t cstride;
    int s_lo, s_n, r_lo, r_n;
};
// Per-row sums of the element blocks (k_rowsum_f32): row i's slots are
// [rowslot[i], rowslot[i+1]) of kslot, its support entries in support order, each
// ceil(m_e / 16) blocks of 16 slots holding the element block's row of the row's
// function; pos gives each slot's position in the row (0xFFFF: padding).
struct RowSrc {
    int64_t n;
    const int32_t* row_ptr;
    const int32_t* rowslot;  // [n+1]
    const uint16_t* pos;
    const float2* kslot;
    int max_n_i;
};
// Batched row sums: block b sums 16 rows of rule blk_rule[b] from row blk_row[b].
struct RowBatch {
    int64_t n_blocks;
    const int32_t* blk_rule;
    const int64_t* blk_row;
    const RowSrc* src;       // device array
    int max_n_i;             // over the rules
};
// Pack construction (rule set-up, k_pack).
enum { PK_TABLE2 = 0, PK_W2E = 1, PK_GAUSS = 2 };
struct PackJob {
    int64_t E;
    int kind, ncomp, nc, nwc;
    const int32_t* m;
    const int32_t* P;
    const int64_t* src_off;  // table offset (PK_TABLE2, PK_GAUSS) or element-major weight row (PK_W2E)
    const int64_t* out_off;
    const int64_t* pt0;      // first Gauss point (PK_GAUSS)
    const float2* f2;
    const double* f64;
    const double* gw;
    float2* out;
};

// (hi, lo) float pair of a double v with hi + lo = v to 2^-47 |v|: hi is v cut to 24
// significant bits, lo the next 24 bits of the remainder (cut as well).  Built from the
// encoding with integer instructions for 2^-60 < |v| < 2^100 (the FP64 conversions run on
// the slow FP64 pipe of this GPU); outside that range, and for 0, by conversions in an
// out-of-line function, so that the common path carries no FP64 instruction (a short
// branch would otherwise be if-converted and every call would issue the conversions).
static __device__ __noinline__ float2 split_double_by_conversion(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ float2 split_double(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ffu) - 1023;
    if (ex <= -60 || ex >= 100) return split_double_by_conversion(v);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;                  // 52 bits
    const float hi = __uint_as_float(sign | ((unsigned)(ex + 127) << 23) | (unsigned)(mant >> 29));
    const unsigned r = (unsigned)(mant & 0x1FFFFFFFu);                      // the other 29 bits
    const int msb = 31 - __clz(r | 1u);                                     // 0..28 (r = 0: lo = 0 below)
    const unsigned m24 = msb >= 23 ? (r >> (msb - 23)) : (r << (23 - msb));  // leading one at bit 23
    const float lo = __uint_as_float(sign | ((unsigned)(ex - 52 + msb + 127) << 23) | (m24 & 0x7FFFFFu));
    return make_float2(hi, r == 0u ? 0.0f : lo);
}

// Per-call device pointers, passed as a kernel parameter (N = 1 for one rule).
constexpr int WQ_BATCH_MAX = 256;
template <int N>
struct PtrTable {
    const double* coef[N];
    float* vals[N];
};

// Several rules assembled by one launch of each kernel: the concatenated tiles
// (item / kb / item_rule), the rules' data (src[k], device), and the blocks of the
// per-entry sums (gblk_rule, gblk_start: 512 entries of one rule per block).
struct BatchPlan {
    int64_t n_items;
    const int4* item;
    const int32_t* kb;
    const int32_t* item_rule;
    const ElemSrc* src;
    int64_t n_gblocks;
    const int32_t* gblk_rule;
    const int64_t* gblk_start;
};

}  // namespace wqd
