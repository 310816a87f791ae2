// Host-side mesh preprocessing of the CGP library (the paper's preprocessing stage, Sect. 2.4):
// validation, nested 1:4 refinement (Sect. 2.2), the s^p / s^u tables (Remark 2.2, Eqs. 29-30),
// P1 CSR patterns, element-to-CSR slot maps and the element colouring used by the assembly.
#pragma once
#include <vector>
#include "cgp.h"

namespace cgp {

struct HostLevel {
    int n = 0, t = 0;
    std::vector<double> xy;   // [n][2]
    std::vector<int> tri;     // [t][3]
};

struct HostCsr {
    int n = 0, nnz = 0;
    std::vector<int> rp, ci, diag;   // row pointers [n+1], sorted columns [nnz], diagonal slot [n]
};

struct HostElems {
    std::vector<int> slot;     // [t][9]: CSR slot of (row tri[a], col tri[b]) at a*3+b
    std::vector<int> perm;     // elements sorted by colour
    std::vector<int> colptr;   // [n_colours+1] offsets into perm
};

struct HostMesh {
    std::vector<HostLevel> lv;               // lv[0] coarse (pressure) ... lv[L] fine (velocity)
    std::vector<std::vector<int>> sp;        // sp[k]: [N_{k+1}][2] parent pair (beta, gamma)
    std::vector<int> su;                     // [N_c] fine index xi of each coarse node
    // Fine-node storage order: fperm[i] is the refinement-order index of stored fine node i
    // (empty: the refinement order itself). Everything of the fine level above (xy, tri, the last
    // s^p table's rows, su, onb_f, the fine CSR and elements) is in the stored order.
    std::vector<int> fperm;
    // Stored order of the fine triangles when fperm is set: tperm[k] is the refinement-order index
    // of stored triangle k (sorted by their smallest stored node index).
    std::vector<int> tperm;
    HostCsr fine, coarse;
    HostElems ef, ec;
    std::vector<unsigned char> onb_f, onb_c; // on-boundary flags
};

// Sliced ELL (SELL-C-sigma) layout of a CSR pattern: rows sorted by decreasing length within
// windows of `sigma` rows, cut into slices of C rows; slice s holds width[s] slots, slot k of
// lane l at ptr[s] + k * C + l. src[p] is the CSR index of slot p (-1 for padding, whose column
// is the row itself); perm[s * C + l] is the CSR row of lane l of slice s (-1 past the end).
struct HostSell {
    int C = 32, nslices = 0;
    std::vector<int> ptr, width, col, src, perm;
};
void build_sell(const HostCsr& c, int C, int sigma, HostSell& out);

// Build everything from a coarse mesh. With renumber_fine (and levels >= 1) the fine nodes are
// stored in Hilbert-curve order of their coordinates (fperm). Returns CGP_OK, CGP_ERR_ARG or
// CGP_ERR_MESH.
int build_host_mesh(const cgp_mesh_desc* d, int levels, HostMesh& out, bool renumber_fine = false);


}  // namespace cgp
