// Test driver for the library's host-side preprocessing (compiled with g++ by
// tests/test_host_logic_cpu.py; no GPU). It reads a coarse mesh from stdin, runs the library's own
// build_host_mesh, build_sell and Schwarz coarse-space routines on it and prints what they build,
// one labelled whitespace-separated array per line, for the test to check against definitions.
//
// stdin:  levels renumber S   /  n_nodes n_tris  /  xy[n][2]  /  tri[t][3]
// stdout: "<name> <count> v0 v1 ..." lines.
#include <cstdio>
#include <string>
#include <type_traits>
#include <vector>

#include "host_mesh.h"
#include "subdomain.h"

namespace {

template <typename T>
void put(const char* name, const std::vector<T>& v) {
    std::printf("%s %zu", name, v.size());
    for (const T& x : v) {
        if constexpr (std::is_floating_point<T>::value) std::printf(" %.17g", (double)x);
        else std::printf(" %lld", (long long)x);
    }
    std::printf("\n");
}

}  // namespace

int main() {
    int levels = 0, renumber = 0, S = 64, n = 0, t = 0;
    if (std::scanf("%d %d %d %d %d", &levels, &renumber, &S, &n, &t) != 5) return 2;
    std::vector<double> xy(2 * (size_t)n);
    std::vector<int> tri(3 * (size_t)t);
    for (auto& v : xy)
        if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : tri)
        if (std::scanf("%d", &v) != 1) return 2;
    cgp_mesh_desc d{n, t, xy.data(), tri.data()};
    cgp::HostMesh H;
    const int st = cgp::build_host_mesh(&d, levels, H, renumber != 0);
    std::printf("status 1 %d\n", st);
    if (st != CGP_OK) return 0;

    // fine level as stored: coordinates, triangles, storage order, CSR, element slots
    const cgp::HostLevel& F = H.lv[levels];
    put("fine_xy", F.xy);
    put("fine_tri", F.tri);
    put("fperm", H.fperm);
    put("fine_rp", H.fine.rp);
    put("fine_ci", H.fine.ci);
    put("fine_diag", H.fine.diag);
    put("fine_slot", H.ef.slot);
    put("coarse_rp", H.coarse.rp);
    put("coarse_ci", H.coarse.ci);
    put("su", H.su);

    // sliced ELL of the fine pattern: sorted in windows of 32 rows (stand-alone product) and in the
    // natural row order (fine solvers)
    for (int sigma : {32, 1}) {
        cgp::HostSell hs;
        cgp::build_sell(H.fine, 32, sigma, hs);
        const std::string tag = "sell" + std::to_string(sigma) + "_";
        put((tag + "ptr").c_str(), hs.ptr);
        put((tag + "width").c_str(), hs.width);
        put((tag + "col").c_str(), hs.col);
        put((tag + "src").c_str(), hs.src);
        put((tag + "perm").c_str(), hs.perm);
    }

    // Schwarz coarse space on the coarse level with the SPD test matrix A = I + graph Laplacian
    // of the coarse pattern: Hilbert renumbering, S-row subdomains, linear functions, A_0^-1
    const cgp::HostLevel& Cl = H.lv[0];
    const cgp::HostCsr& C = H.coarse;
    std::vector<double> v(C.nnz);
    for (int i = 0; i < C.n; ++i)
        for (int k = C.rp[i]; k < C.rp[i + 1]; ++k)
            v[k] = C.ci[k] == i ? 1.0 + (C.rp[i + 1] - C.rp[i] - 1) : -1.0;
    const std::vector<int> perm = cgp::hilbert_order(Cl.xy, C.n);
    std::vector<int> inv(C.n);
    for (int i = 0; i < C.n; ++i) inv[perm[i]] = i;
    std::vector<int> rp2(C.n + 1, 0), ci2;
    std::vector<double> v2;
    for (int i = 0; i < C.n; ++i) {
        const int r = perm[i];
        for (int k = C.rp[r]; k < C.rp[r + 1]; ++k) {
            ci2.push_back(inv[C.ci[k]]);
            v2.push_back(v[k]);
        }
        rp2[i + 1] = (int)ci2.size();
    }
    const int nsub = (C.n + S - 1) / S;
    const std::vector<int> sub = cgp::chunk_subdomains(C.n, S);
    const std::vector<double> fxy = cgp::linear_functions(Cl.xy, perm, sub, C.n, nsub);
    std::vector<double> Ai;
    const int gs = cgp::galerkin_inverse(rp2, ci2, v2, fxy, sub, C.n, nsub, Ai);
    std::printf("galerkin_status 1 %d\n", gs);
    put("schwarz_perm", perm);
    put("schwarz_sub", sub);
    put("schwarz_fxy", fxy);
    put("schwarz_Ai", Ai);
    return 0;
}
