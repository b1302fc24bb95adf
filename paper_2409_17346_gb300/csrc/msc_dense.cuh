// Dense discrete gradient of a whole 3D field, one z-slab of a 32 x TY anchor tile per block.
//
// The per-anchor evaluator (eval_anchor) recomputes, for every anchor, the vertex pairs of
// the 8 corners of its cube and the pairings of the 19 cube edges and 18 cube triangles that
// its own cells depend on.  Over a whole field that repeats each vertex pair 8 times and each
// edge and triangle pairing about twice.  This kernel computes every pairing once per tile
// instead, level by level, as the pairing rules of Sec. 4.2 depend on one another:
//   vertex pair (lowest lower neighbour)  <-  values
//   edge: paired down with its higher vertex, else up with the lowest cofacet below it
//                                         <-  vertex pairs of both ends, values
//   triangle: paired down with its highest edge, else up  <-  edge pairings, values
//   tetrahedron: paired down with its highest triangle     <-  triangle pairings, values
// A block marches up its slab of z-planes: at step j it loads value plane z0+j+1 and computes
// vertex pairs of plane z0+j, edges of z0+j-1, triangles of z0+j-2 and the codes (tetrahedra)
// of z0+j-3, each level over the tile grown by the reach of the next level.  Planes live in
// shared-memory rings just deep enough for their last reader.  The codes equal eval_anchor's
// bit for bit: the same comparisons in the same candidate order, +inf outside the domain.
#pragma once
#include "msc_cells.cuh"

namespace msc {
namespace dense {

// Tile shapes: 32 anchors along x (a warp per row, so the per-warp ballots of the mismatch
// bits cover whole rows) by TY rows, one block of 32 * TY threads, marching up ZS planes.
// The autotuner in the library times the instantiated shapes per grid and keeps the fastest;
// every shape gives the same codes.
template <int TY_, int ZS_> struct Tile {
    static constexpr int TX = 32, TY = TY_, ZS = ZS_, NT = 32 * TY_;
    static constexpr int VX = TX + 5, VY = TY + 5;   // values: x0-1 .. x0+TX+3
    static constexpr int PX = TX + 3, PY = TY + 3;   // vertex pairs: x0 .. x0+TX+2
    static constexpr int EX = TX + 2, EY = TY + 2;   // edges: x0 .. x0+TX+1
    static constexpr int RX = TX + 1, RY = TY + 1;   // triangles: x0 .. x0+TX
};
constexpr int NVAL = 5, NVP = 4, NEDG = 3, NTRI = 2;   // ring depths

constexpr bool pos_lt(const int *a, const int *b)   // vertex-id order of two offsets
{
    return a[2] != b[2] ? a[2] < b[2] : (a[1] != b[1] ? a[1] < b[1] : a[0] < b[0]);
}

struct Tabs {
    int vord[14];                     // neighbour indices by increasing vertex id
    int e_b[7][3];                    // edge type e: offset of its upper vertex
    int e_nc[7];
    int e_c[7][6][3];                 //   cofacet candidates (vertex-id order)
    unsigned e_lta[7], e_ltb[7];      //   candidate i has a smaller id than vertex a / b
    int t_v[12][3][3];                // triangle type: vertex offsets (slot 0, 1, 2 = 0, A, B)
    int t_he[12][3][3];               //   highest edge when slot j is lowest: anchor offset
    int t_het[12][3], t_hew[12][3];   //   its type, and the cofacet index that means "this triangle"
    int t_c[12][2][3];                //   tetrahedron candidates
    unsigned t_lt[12][3];             //   candidate i has a smaller id than vertex slot j
    int k_v[6][4][3];                 // tetrahedron type: corner offsets (0, kA, kB, 7)
    int k_f[6][4][3], k_ft[6][4], k_fw[6][4];   // facet opposite corner slot j, its cofacet index
};

constexpr Tabs make_tabs()
{
    constexpr Tab<3> T = make_tab<3>();
    Tabs d{};
    for (int i = 0; i < 14; i++) d.vord[i] = T.cnb_ord[0][i];
    for (int e = 0; e < 7; e++) {
        const int A = e + 1;
        const int b[3] = {A & 1, (A >> 1) & 1, (A >> 2) & 1}, a[3] = {0, 0, 0};
        for (int k = 0; k < 3; k++) d.e_b[e][k] = b[k];
        d.e_nc[e] = T.necof[e];
        for (int i = 0; i < T.necof[e]; i++) {
            for (int k = 0; k < 3; k++) d.e_c[e][i][k] = T.ecof_v[e][i][k];
            if (pos_lt(T.ecof_v[e][i], a)) d.e_lta[e] |= 1u << i;
            if (pos_lt(T.ecof_v[e][i], b)) d.e_ltb[e] |= 1u << i;
        }
    }
    for (int t = 0; t < 12; t++) {
        const int A = T.tA[t], B = T.tB[t];
        const int cs[3] = {0, A, B};
        for (int j = 0; j < 3; j++) {
            d.t_v[t][j][0] = cs[j] & 1; d.t_v[t][j][1] = (cs[j] >> 1) & 1; d.t_v[t][j][2] = (cs[j] >> 2) & 1;
        }
        // slot j lowest: the highest edge is the one opposite it; its cofacet list holds the
        // vertex of slot j at the position that means this triangle
        for (int j = 0; j < 3; j++) {
            int q = 0;
            for (int r = 0; r < 3; r++) if (T.tfac_opp[t][r] == cs[j]) q = r;
            const int et = T.tfac_type[t][q];
            for (int k = 0; k < 3; k++) d.t_he[t][j][k] = T.tfac_anc[t][q][k];
            d.t_het[t][j] = et;
            int w = -1;
            for (int i = 0; i < T.necof[et]; i++) {
                bool eq = true;
                for (int k = 0; k < 3; k++) eq = eq && T.ecof_v[et][i][k] == d.t_v[t][j][k] - T.tfac_anc[t][q][k];
                if (eq) w = i;
            }
            d.t_hew[t][j] = w;
        }
        for (int i = 0; i < 2; i++) {
            for (int k = 0; k < 3; k++) d.t_c[t][i][k] = T.tcof_v[t][i][k];
            for (int j = 0; j < 3; j++)
                if (pos_lt(T.tcof_v[t][i], d.t_v[t][j])) d.t_lt[t][j] |= 1u << i;
        }
    }
    for (int k = 0; k < 6; k++) {
        const int cs[4] = {0, T.kA[k], T.kB[k], 7};
        for (int j = 0; j < 4; j++) {
            d.k_v[k][j][0] = cs[j] & 1; d.k_v[k][j][1] = (cs[j] >> 1) & 1; d.k_v[k][j][2] = (cs[j] >> 2) & 1;
        }
        for (int j = 0; j < 4; j++) {
            const int ft = T.kfac_type[k][j];
            for (int q = 0; q < 3; q++) d.k_f[k][j][q] = T.kfac_anc[k][j][q];
            d.k_ft[k][j] = ft;
            int w = -1;
            for (int i = 0; i < T.ntcof[ft]; i++) {
                bool eq = true;
                for (int q = 0; q < 3; q++) eq = eq && T.tcof_v[ft][i][q] == d.k_v[k][j][q] - T.kfac_anc[k][j][q];
                if (eq) w = i;
            }
            d.k_fw[k][j] = w;
        }
    }
    return d;
}

struct TabsC {
    static constexpr Tabs D = make_tabs();
};

// reach of the rules, checked against the plane ring and the region margins
constexpr bool reach_ok()
{
    constexpr Tabs d = make_tabs();
    for (int e = 0; e < 7; e++)
        for (int i = 0; i < d.e_nc[e]; i++)
            for (int k = 0; k < 3; k++)
                if (d.e_c[e][i][k] < -1 || d.e_c[e][i][k] > 2) return false;
    for (int t = 0; t < 12; t++)
        for (int i = 0; i < 2; i++)
            for (int k = 0; k < 3; k++)
                if (d.t_c[t][i][k] < -1 || d.t_c[t][i][k] > 2) return false;
    for (int t = 0; t < 12; t++)
        for (int j = 0; j < 3; j++) {
            if (d.t_hew[t][j] < 0) return false;
            for (int k = 0; k < 3; k++) if (d.t_he[t][j][k] < 0 || d.t_he[t][j][k] > 1) return false;
        }
    for (int k = 0; k < 6; k++)
        for (int j = 0; j < 4; j++) {
            if (d.k_fw[k][j] < 0) return false;
            for (int q = 0; q < 3; q++) if (d.k_f[k][j][q] < 0 || d.k_f[k][j][q] > 1) return false;
        }
    return true;
}
static_assert(reach_ok(), "pairing rule reach exceeds the dense tile's margins");

template <class TL> struct Smem {
    float val[NVAL][TL::VY][TL::VX];
    uint8_t vp[NVP][TL::PY][TL::PX];
    uint32_t ef[NEDG][TL::EY][TL::EX];
    uint32_t tf[NTRI][TL::RY][TL::RX];
};

}  // namespace dense
}  // namespace msc
