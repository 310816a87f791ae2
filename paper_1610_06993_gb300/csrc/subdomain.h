// Host-side construction of the subdomain coarse spaces of the two-level Schwarz preconditioners
// (krylov_pipe.cu: one subdomain per block of the on-chip kernel; krylov_2l.cu: fixed 256-row
// subdomains of the batched kernel). Nodes are renumbered along a Hilbert curve so that
// contiguous row ranges are compact patches; each subdomain contributes three coarse functions,
// the restrictions of 1, (x - xbar) / H and (y - ybar) / H (centroid and RMS radius of its
// nodes); the Galerkin matrix A_0 = R_0 A R_0^T is inverted by Cholesky factorisation.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "cgp.h"

namespace cgp {

#define SZ_NC 3   // coarse functions per subdomain

// Position of the cell (x, y), 0 <= x, y < 2^bits, along the Hilbert curve. At each scale the
// quadrant of the point gives two digits of the position; the remaining low bits are then
// reflected and transposed into the orientation of that quadrant's sub-curve (complementing all
// bits reflects the low bits, which are the only ones read afterwards).
inline uint64_t hilbert_index(uint32_t x, uint32_t y, int bits) {
    uint64_t d = 0;
    for (int k = bits - 1; k >= 0; --k) {
        const uint32_t s = 1u << k;
        const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = ~x;
                y = ~y;
            }
            std::swap(x, y);
        }
    }
    return d;
}

// Nodes in Hilbert-curve order of their coordinates xy[n][2] (one scale for both axes, so a
// row range is compact in physical space); ties keep the original order.
inline std::vector<int> hilbert_order(const std::vector<double>& xy, int n) {
    double x0 = xy[0], x1 = xy[0], y0 = xy[1], y1 = xy[1];
    for (int i = 0; i < n; ++i) {
        x0 = std::min(x0, xy[2 * i]);
        x1 = std::max(x1, xy[2 * i]);
        y0 = std::min(y0, xy[2 * i + 1]);
        y1 = std::max(y1, xy[2 * i + 1]);
    }
    const double ext = std::max(x1 - x0, y1 - y0);
    const double sc = ext > 0.0 ? 65535.0 / ext : 0.0;
    std::vector<uint64_t> key(n);
    for (int i = 0; i < n; ++i) {
        const uint32_t hx = (uint32_t)std::min(65535.0, std::max(0.0, (xy[2 * i] - x0) * sc));
        const uint32_t hy = (uint32_t)std::min(65535.0, std::max(0.0, (xy[2 * i + 1] - y0) * sc));
        key[i] = hilbert_index(hx, hy, 16);
    }
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int p, int q) { return key[p] < key[q]; });
    return perm;
}

// Subdomain of every renumbered row for subdomains of S consecutive rows (the last may be shorter).
inline std::vector<int> chunk_subdomains(int n, int S) {
    std::vector<int> sub(n);
    for (int i = 0; i < n; ++i) sub[i] = i / S;
    return sub;
}

// The two linear coarse functions at every renumbered node (fxy[2 i], fxy[2 i + 1]), for the
// subdomain sub[i] of each renumbered row (nsub subdomains; an empty one has no functions).
inline std::vector<double> linear_functions(const std::vector<double>& xy, const std::vector<int>& perm,
                                            const std::vector<int>& sub, int n, int nsub) {
    std::vector<double> mx(nsub, 0.0), my(nsub, 0.0), h2(nsub, 0.0), cnt(nsub, 0.0), f(2 * (size_t)n, 0.0);
    for (int i = 0; i < n; ++i) {
        mx[sub[i]] += xy[2 * perm[i]];
        my[sub[i]] += xy[2 * perm[i] + 1];
        cnt[sub[i]] += 1.0;
    }
    for (int a = 0; a < nsub; ++a)
        if (cnt[a] > 0.0) {
            mx[a] /= cnt[a];
            my[a] /= cnt[a];
        }
    for (int i = 0; i < n; ++i) {
        const double dx = xy[2 * perm[i]] - mx[sub[i]], dy = xy[2 * perm[i] + 1] - my[sub[i]];
        h2[sub[i]] += dx * dx + dy * dy;
    }
    for (int i = 0; i < n; ++i) {
        const int a = sub[i];
        const double ih = h2[a] > 0.0 ? 1.0 / std::sqrt(h2[a] / cnt[a]) : 0.0;
        f[2 * (size_t)i] = (xy[2 * perm[i]] - mx[a]) * ih;
        f[2 * (size_t)i + 1] = (xy[2 * perm[i] + 1] - my[a]) * ih;
    }
    return f;
}

// Inverse of the Galerkin coarse matrix for the subdomains sub[i] of the rows of the renumbered
// CSR matrix (rp, ci, v): coarse index of function f on subdomain a is f * nsub + a. A coarse
// function that vanishes on its subdomain gets a unit diagonal and no coupling. Returns CGP_OK,
// or CGP_ERR_ARG if the matrix is not positive definite on the coarse space.
inline int galerkin_inverse(const std::vector<int>& rp, const std::vector<int>& ci, const std::vector<double>& v,
                            const std::vector<double>& fxy, const std::vector<int>& sub, int n, int nsub,
                            std::vector<double>& Ai) {
    const int nc0 = SZ_NC * nsub;
    std::vector<double> A0((size_t)nc0 * nc0, 0.0), Lc((size_t)nc0 * nc0, 0.0);
    Ai.assign((size_t)nc0 * nc0, 0.0);
    for (int i = 0; i < n; ++i) {
        const double pi[SZ_NC] = {1.0, fxy[2 * (size_t)i], fxy[2 * (size_t)i + 1]};
        const int ai = sub[i];
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k], aj = sub[j];
            const double pj[SZ_NC] = {1.0, fxy[2 * (size_t)j], fxy[2 * (size_t)j + 1]};
            for (int f = 0; f < SZ_NC; ++f)
                for (int g = 0; g < SZ_NC; ++g)
                    A0[(size_t)(f * nsub + ai) * nc0 + g * nsub + aj] += pi[f] * v[k] * pj[g];
        }
    }
    for (int q = 0; q < nc0; ++q)
        if (A0[(size_t)q * nc0 + q] == 0.0) A0[(size_t)q * nc0 + q] = 1.0;
    for (int j = 0; j < nc0; ++j) {
        double d = A0[(size_t)j * nc0 + j];
        for (int k = 0; k < j; ++k) d -= Lc[(size_t)j * nc0 + k] * Lc[(size_t)j * nc0 + k];
        if (!(d > 0.0)) return CGP_ERR_ARG;
        const double ljj = std::sqrt(d);
        Lc[(size_t)j * nc0 + j] = ljj;
        for (int i = j + 1; i < nc0; ++i) {
            double s = A0[(size_t)i * nc0 + j];
            for (int k = 0; k < j; ++k) s -= Lc[(size_t)i * nc0 + k] * Lc[(size_t)j * nc0 + k];
            Lc[(size_t)i * nc0 + j] = s / ljj;
        }
    }
    // A_0^-1 = Y^T Y with Y = L^-1: rows of Y by axpys of earlier rows (row-major, contiguous)
    std::vector<double> Y((size_t)nc0 * nc0, 0.0);
    for (int i = 0; i < nc0; ++i) {
        double* yi = &Y[(size_t)i * nc0];
        yi[i] = 1.0;
        for (int k = 0; k < i; ++k) {
            const double lik = Lc[(size_t)i * nc0 + k];
            if (lik == 0.0) continue;
            const double* yk = &Y[(size_t)k * nc0];
            for (int j = 0; j <= k; ++j) yi[j] -= lik * yk[j];
        }
        const double inv = 1.0 / Lc[(size_t)i * nc0 + i];
        for (int j = 0; j <= i; ++j) yi[j] *= inv;
    }
    for (int i = 0; i < nc0; ++i) {
        const double* yi = &Y[(size_t)i * nc0];
        for (int a = 0; a <= i; ++a) {
            const double ya = yi[a];
            if (ya == 0.0) continue;
            double* ra = &Ai[(size_t)a * nc0];
            for (int c = 0; c <= a; ++c) ra[c] += ya * yi[c];
        }
    }
    for (int a = 0; a < nc0; ++a)
        for (int c = 0; c < a; ++c) Ai[(size_t)c * nc0 + a] = Ai[(size_t)a * nc0 + c];
    return CGP_OK;
}

}  // namespace cgp
