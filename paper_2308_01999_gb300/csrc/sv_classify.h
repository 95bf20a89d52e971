// sv_classify.h -- exact structure analysis of a gate matrix (host).
//
// Sec. II-D-1 and Table I: diagonal and generalized-permutation gates have a
// lower arithmetic intensity than dense ones and get their own kernels. The
// analysis compares matrix entries exactly (no tolerance), so every rewrite
// below leaves the operator unchanged:
//   * a target bit whose off-diagonal blocks are zero and one of whose
//     diagonal blocks is the identity becomes a control;
//   * a matrix with zero off-diagonal entries is diagonal;
//   * a matrix with one nonzero per row and per column is a generalized
//     permutation.
#pragma once

#include <algorithm>
#include <complex>
#include <vector>

namespace svc {

using cd = std::complex<double>;

struct Gate {
    std::vector<int> t;      // targets, bit j of the matrix index is t[j]
    std::vector<int> c;      // controls
    std::vector<int> cv;     // control values
    std::vector<cd> m;       // 2^k x 2^k row-major
};

inline int ins_bit(int a, int j, int b) {   // insert bit value b at position j of a
    const int lo = a & ((1 << j) - 1);
    return ((a >> j) << (j + 1)) | (b << j) | lo;
}

// If target bit j splits M into blocks with zero off-diagonal blocks and one
// diagonal block equal to the identity, that bit acts as a control: return the
// control value (1 if the bit-0 block is the identity) and the other block.
inline int extract_control(const Gate &g, int j, std::vector<cd> &rest) {
    const int k = (int)g.t.size(), D = 1 << k, H = D / 2;
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c)
            if (((r >> j) & 1) != ((c >> j) & 1) && g.m[r * D + c] != cd(0)) return -1;
    for (int val = 0; val < 2; ++val) {
        bool ident = true;
        for (int a = 0; a < H && ident; ++a)
            for (int b = 0; b < H && ident; ++b)
                if (g.m[ins_bit(a, j, val) * D + ins_bit(b, j, val)] != (a == b ? cd(1) : cd(0))) ident = false;
        if (ident) {
            rest.assign(H * H, cd(0));
            for (int a = 0; a < H; ++a)
                for (int b = 0; b < H; ++b) rest[a * H + b] = g.m[ins_bit(a, j, 1 - val) * D + ins_bit(b, j, 1 - val)];
            return 1 - val;
        }
    }
    return -1;
}

inline void simplify_controls(Gate &g) {
    bool changed = true;
    while (changed && !g.t.empty()) {
        changed = false;
        for (int j = 0; j < (int)g.t.size(); ++j) {
            std::vector<cd> rest;
            const int val = extract_control(g, j, rest);
            if (val < 0) continue;
            g.c.push_back(g.t[j]);
            g.cv.push_back(val);
            g.t.erase(g.t.begin() + j);
            g.m.swap(rest);
            changed = true;
            break;
        }
    }
}

// matrix for targets sorted ascending (new bit i <-> old bit sigma[i])
inline void sort_targets(Gate &g) {
    const int k = (int)g.t.size(), D = 1 << k;
    std::vector<int> sigma(k);
    for (int i = 0; i < k; ++i) sigma[i] = i;
    std::sort(sigma.begin(), sigma.end(), [&](int a, int b) { return g.t[a] < g.t[b]; });
    bool ident = true;
    for (int i = 0; i < k; ++i) ident &= sigma[i] == i;
    if (ident) return;
    auto old_index = [&](int rn) {
        int ro = 0;
        for (int i = 0; i < k; ++i)
            if ((rn >> i) & 1) ro |= 1 << sigma[i];
        return ro;
    };
    std::vector<cd> m2(D * D);
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) m2[r * D + c] = g.m[old_index(r) * D + old_index(c)];
    std::vector<int> t2(k);
    for (int i = 0; i < k; ++i) t2[i] = g.t[sigma[i]];
    g.t.swap(t2);
    g.m.swap(m2);
}


// true if every off-diagonal entry is exactly zero
inline bool is_diagonal(const Gate &g) {
    const int D = 1 << (int)g.t.size();
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c)
            if (r != c && g.m[r * D + c] != cd(0)) return false;
    return true;
}

// one nonzero per row and per column: out[j] = d[j] * in[perm[j]]
inline bool as_permutation(const Gate &g, std::vector<int> &perm, std::vector<cd> &d) {
    const int D = 1 << (int)g.t.size();
    perm.assign(D, -1);
    d.assign(D, cd(0));
    std::vector<int> colcount(D, 0);
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c)
            if (g.m[r * D + c] != cd(0)) {
                if (perm[r] >= 0) return false;
                perm[r] = c;
                d[r] = g.m[r * D + c];
                ++colcount[c];
            }
    for (int j = 0; j < D; ++j)
        if (perm[j] < 0 || colcount[j] != 1) return false;
    return true;
}

}  // namespace svc
