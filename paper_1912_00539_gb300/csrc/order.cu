// Orderings of the cell graph (Sec. 5): reverse Cuthill-McKee, one-way
// dissection, line ordering and the hybrid line-RCM / line-1WD orderings.
// Host code: the orderings are computed once per grid, before any value of
// the matrix is known to the solver, on the pattern in host memory.
//
//  * RCM: breadth-first search from a pseudo-peripheral cell (the last level's
//    lowest-degree cell, ties to the lowest index, repeated while the number
//    of levels grows), neighbours in increasing (degree, index), the order
//    reversed; one component after another (in order of their lowest cell),
//    each reversed on its own.  Degrees are those of the whole graph.
//  * 1WD (one-way dissection): a rooted level structure from a
//    pseudo-peripheral cell; level sets at regular intervals delta are taken as
//    separators (delta = sqrt((3 w + 13) / 2), w the mean level width, the
//    spacing George derived for grids); the cells between separators form
//    independent blocks, numbered first (each block by RCM), and the separator
//    cells last, level by level.
//  * Lines (Sec. 5.1): strongly coupled cells are chained into lines.  A cell
//    is anisotropic when its strongest coupling exceeds its weakest by more
//    than `threshold`.  Starting from the most anisotropic cell not yet in a
//    line, a line grows at each end to the free neighbour with the strongest
//    coupling while that coupling exceeds `threshold` times the end cell's
//    weakest coupling and is within `threshold` of the neighbour's strongest.
//    A cell with no weak coupling (e.g. on a side boundary, where the weak
//    direction has no neighbour) is measured against the weakest coupling of
//    the line's last anisotropic cell, at most two such cells in a row (a
//    third one in a row ends the line); lines of one cell are not lines.  Couplings are per-block weights: the caller's
//    (geometric) weights, or the Frobenius norms of the blocks.
//  * LINE: every line's cells made contiguous, in line order, at the position
//    of the line's first cell in the input order.  LINE_RCM / LINE_1WD: the
//    graph whose vertices are the lines and the cells in no line (two vertices
//    joined when any of their cells are neighbours, Sec. 5.2) is ordered by RCM
//    or 1WD and each line expanded in place.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace abilu {
namespace order {

struct Graph {  // symmetric adjacency without self loops
    int n;
    std::vector<int> ptr, adj;
};

static Graph from_pattern(int n, const int32_t *rowptr, const int32_t *colind) {
    // symmetrise: an edge i - j when either block (i,j) or (j,i) is present
    std::vector<std::pair<int, int>> e;
    e.reserve((size_t)rowptr[n] * 2);
    for (int i = 0; i < n; i++)
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const int j = colind[p];
            if (j == i) continue;
            e.emplace_back(i, j);
            e.emplace_back(j, i);
        }
    std::sort(e.begin(), e.end());
    e.erase(std::unique(e.begin(), e.end()), e.end());
    Graph g;
    g.n = n;
    g.ptr.assign(n + 1, 0);
    for (auto &x : e) g.ptr[x.first + 1]++;
    for (int i = 0; i < n; i++) g.ptr[i + 1] += g.ptr[i];
    g.adj.resize(e.size());
    for (size_t k = 0; k < e.size(); k++) g.adj[k] = e[k].second;  // sorted by (i, j)
    return g;
}

static inline int degree(const Graph &g, int v) { return g.ptr[v + 1] - g.ptr[v]; }

// BFS levels from `root` over the cells with mask[c] == tag; returns the
// cells in BFS order and fills level[] (-1 elsewhere is the caller's job)
static std::vector<int> bfs(const Graph &g, int root, const std::vector<int> &mask, int tag,
                            std::vector<int> &level, int *nlev) {
    std::vector<int> out{root};
    level[root] = 0;
    int lv = 0;
    for (size_t h = 0; h < out.size(); h++) {
        const int v = out[h];
        lv = level[v];
        for (int p = g.ptr[v]; p < g.ptr[v + 1]; p++) {
            const int u = g.adj[p];
            if (mask[u] == tag && level[u] < 0) {
                level[u] = level[v] + 1;
                out.push_back(u);
            }
        }
    }
    *nlev = lv + 1;
    return out;
}

// pseudo-peripheral cell of the component of `start` (cells with mask == tag):
// from the root's level structure, the last level's cell of least degree (ties:
// lowest index) becomes the root while its level structure is deeper (the
// number of levels grows strictly and is at most the component's size, so
// the loop ends)
static int pseudo_peripheral(const Graph &g, int start, const std::vector<int> &mask, int tag,
                             std::vector<int> &level) {
    int root = start, nlev = 0;
    for (;;) {
        std::vector<int> comp = bfs(g, root, mask, tag, level, &nlev);
        int best = -1;
        for (int v : comp)
            if (level[v] == nlev - 1 &&
                (best < 0 || degree(g, v) < degree(g, best) ||
                 (degree(g, v) == degree(g, best) && v < best)))
                best = v;
        int nlev2 = 0;
        for (int v : comp) level[v] = -1;
        std::vector<int> comp2 = bfs(g, best, mask, tag, level, &nlev2);
        for (int v : comp2) level[v] = -1;
        if (nlev2 <= nlev) return root;
        root = best;
    }
}

// Cuthill-McKee order of the component of `start` (mask == tag), appended to out
static void cuthill_mckee(const Graph &g, int start, const std::vector<int> &mask, int tag,
                          std::vector<int> &level, std::vector<int> &out) {
    const int root = pseudo_peripheral(g, start, mask, tag, level);
    const size_t o0 = out.size();
    out.push_back(root);
    level[root] = 0;
    std::vector<int> nb;
    for (size_t h = o0; h < out.size(); h++) {
        const int v = out[h];
        nb.clear();
        for (int p = g.ptr[v]; p < g.ptr[v + 1]; p++) {
            const int u = g.adj[p];
            if (mask[u] == tag && level[u] < 0) {
                level[u] = level[v] + 1;
                nb.push_back(u);
            }
        }
        std::sort(nb.begin(), nb.end(), [&](int a, int b) {
            return degree(g, a) != degree(g, b) ? degree(g, a) < degree(g, b) : a < b;
        });
        out.insert(out.end(), nb.begin(), nb.end());
    }
}

// RCM of every component of the cells with mask == tag, in order of their
// lowest cell; each component reversed on its own
static void rcm(const Graph &g, const std::vector<int> &mask, int tag, std::vector<int> &level,
                std::vector<int> &out) {
    for (int s = 0; s < g.n; s++) {
        if (mask[s] != tag || level[s] >= 0) continue;
        const size_t o0 = out.size();
        cuthill_mckee(g, s, mask, tag, level, out);
        std::reverse(out.begin() + (long)o0, out.end());
    }
}

// one-way dissection of every component of the cells with mask == tag
static void one_way(const Graph &g, std::vector<int> &mask, int tag, std::vector<int> &level,
                    std::vector<int> &out) {
    std::vector<int> seps;
    for (int s = 0; s < g.n; s++) {
        if (mask[s] != tag || level[s] >= 0) continue;
        const int root = pseudo_peripheral(g, s, mask, tag, level);
        int nlev = 0;
        std::vector<int> comp = bfs(g, root, mask, tag, level, &nlev);
        const double w = (double)comp.size() / nlev;
        const int delta = std::max(2, (int)lround(sqrt((3.0 * w + 13.0) / 2.0)));
        if (nlev < 2 * delta + 1) {  // too shallow to dissect: RCM of the component
            for (int v : comp) level[v] = -1;
            const size_t o0 = out.size();
            cuthill_mckee(g, s, mask, tag, level, out);
            std::reverse(out.begin() + (long)o0, out.end());
            continue;
        }
        // separator levels delta, 2 delta, ... (< nlev - 1): marked with tag+1
        const int septag = tag + 1;
        std::vector<int> sep_lv;
        for (int l = delta; l < nlev - 1; l += delta) sep_lv.push_back(l);
        std::vector<char> is_sep(nlev, 0);
        for (int l : sep_lv) is_sep[l] = 1;
        std::vector<int> sep_cells;
        for (int v : comp) {
            if (is_sep[level[v]]) {
                mask[v] = septag;
                sep_cells.push_back(v);
            }
        }
        // blocks: components of the rest, each by RCM
        for (int v : comp) level[v] = -1;
        for (int v : comp) {
            if (mask[v] != tag || level[v] >= 0) continue;
            const size_t o0 = out.size();
            cuthill_mckee(g, v, mask, tag, level, out);
            std::reverse(out.begin() + (long)o0, out.end());
        }
        // separators last, level by level (comp is in BFS order)
        for (int v : sep_cells) {
            level[v] = 0;   // visited
            seps.push_back(v);
        }
    }
    out.insert(out.end(), seps.begin(), seps.end());
}

// lines of strongly coupled cells: line_of[v] = line index or -1
static int find_lines(const Graph &g, const int32_t *rowptr, const int32_t *colind,
                      const double *wblk, double threshold, std::vector<int> &line_of,
                      std::vector<std::vector<int>> &lines) {
    const int n = g.n;
    // symmetric coupling per graph edge: max of the two block weights
    std::vector<double> wadj(g.adj.size(), 0.0);
    auto slot = [&](int i, int j) -> long {
        const int *b = g.adj.data() + g.ptr[i], *e = g.adj.data() + g.ptr[i + 1];
        const int *f = std::lower_bound(b, e, j);
        return (f != e && *f == j) ? (long)(f - g.adj.data()) : -1;
    };
    for (int i = 0; i < n; i++)
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const int j = colind[p];
            if (j == i) continue;
            const long a = slot(i, j), b = slot(j, i);
            wadj[a] = std::max(wadj[a], wblk[p]);
            wadj[b] = std::max(wadj[b], wblk[p]);
        }
    std::vector<double> wmax(n, 0.0), wmin(n, 0.0), aniso(n, 1.0);
    for (int i = 0; i < n; i++) {
        double mx = 0.0, mn = INFINITY;
        for (int p = g.ptr[i]; p < g.ptr[i + 1]; p++) {
            mx = std::max(mx, wadj[p]);
            mn = std::min(mn, wadj[p]);
        }
        wmax[i] = mx;
        wmin[i] = g.ptr[i + 1] > g.ptr[i] ? mn : 0.0;
        aniso[i] = (mn > 0.0 && mn < INFINITY) ? mx / mn : (mx > 0.0 ? INFINITY : 1.0);
    }
    std::vector<int> seeds(n);
    std::iota(seeds.begin(), seeds.end(), 0);
    std::stable_sort(seeds.begin(), seeds.end(), [&](int a, int b) { return aniso[a] > aniso[b]; });
    line_of.assign(n, -1);
    lines.clear();
    // Strongest free neighbour of the line's end c, if the edge continues the
    // line: strong against `ref` (c's weakest coupling, or for a cell with no
    // weak coupling -- e.g. on a side boundary -- the weakest coupling of the
    // line's last anisotropic cell) and among the neighbour's strongest.
    auto next = [&](int c, double ref) {
        int best = -1;
        double bw = -1.0;
        for (int p = g.ptr[c]; p < g.ptr[c + 1]; p++) {
            const int u = g.adj[p];
            if (line_of[u] >= 0) continue;
            if (wadj[p] > bw) { bw = wadj[p]; best = u; }
        }
        if (best < 0) return -1;
        if (bw < threshold * ref || bw * threshold < wmax[best]) return -1;
        return best;
    };
    constexpr int MAX_PLAIN_RUN = 2;   // cells without a weak coupling in a row
    auto grow = [&](int s, int id, std::vector<int> &cells) {
        double ref = wmin[s];
        int run = 0;
        for (int c = s;;) {
            const bool an = aniso[c] >= threshold;
            const int u = next(c, an ? wmin[c] : ref);
            if (u < 0) break;
            if (aniso[u] < threshold && run >= MAX_PLAIN_RUN) break;   // a third in a row
            line_of[u] = id;
            cells.push_back(u);
            if (aniso[u] >= threshold) {
                ref = wmin[u];
                run = 0;
            } else {
                run++;
            }
            c = u;
        }
    };
    for (int s : seeds) {
        if (aniso[s] < threshold) break;
        if (line_of[s] >= 0) continue;
        const int id = (int)lines.size();
        std::vector<int> fwd{s}, bwd;
        line_of[s] = id;
        grow(s, id, fwd);
        grow(s, id, bwd);
        if (fwd.size() + bwd.size() < 2) {  // a single cell is not a line
            line_of[s] = -1;
            continue;
        }
        std::vector<int> line(bwd.rbegin(), bwd.rend());
        line.insert(line.end(), fwd.begin(), fwd.end());
        lines.push_back(std::move(line));
    }
    // renumber lines in order of their lowest cell, so the result does not
    // depend on ties in the anisotropy ranking beyond the lines themselves
    std::vector<int> idx(lines.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::vector<int> lo(lines.size());
    for (size_t k = 0; k < lines.size(); k++) lo[k] = *std::min_element(lines[k].begin(), lines[k].end());
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return lo[a] < lo[b]; });
    std::vector<std::vector<int>> sorted(lines.size());
    for (size_t k = 0; k < idx.size(); k++) {
        sorted[k] = std::move(lines[idx[k]]);
        for (int v : sorted[k]) line_of[v] = (int)k;
    }
    lines = std::move(sorted);
    return (int)lines.size();
}

}  // namespace order
}  // namespace abilu

using namespace abilu;
using namespace abilu::order;

extern "C" abilu_status abilu_order(int32_t n, const int32_t *rowptr, const int32_t *colind,
                                    const double *weights, const double *vals, int32_t kind,
                                    double line_threshold, int32_t *perm, int32_t *line_of_out) {
    if (n < 1 || !rowptr || !colind || !perm) return fail(ABILU_EINVAL, "order: bad argument");
    if (rowptr[0] != 0) return fail(ABILU_EINVAL, "order: rowptr[0] must be 0");
    for (int i = 0; i < n; i++)
        if (rowptr[i + 1] < rowptr[i]) return fail(ABILU_EINVAL, "order: rowptr decreasing at %d", i);
    const int64_t nnzb = rowptr[n];
    for (int64_t p = 0; p < nnzb; p++)
        if (colind[p] < 0 || colind[p] >= n) return fail(ABILU_EINVAL, "order: column out of range");
    const bool lined = kind == ABILU_ORDER_LINE || kind == ABILU_ORDER_LINE_RCM ||
                       kind == ABILU_ORDER_LINE_1WD;
    if (kind < ABILU_ORDER_RCM || kind > ABILU_ORDER_LINE_1WD) return fail(ABILU_EINVAL, "order: bad kind");
    if (lined && !weights && !vals) return fail(ABILU_EINVAL, "order: line orderings need weights or values");
    if (lined && !(line_threshold > 1.0)) return fail(ABILU_EINVAL, "order: line threshold must exceed 1");
    Graph g = from_pattern(n, rowptr, colind);
    std::vector<int> level(n, -1), out;
    out.reserve(n);
    std::vector<int> line_of(n, -1);
    if (kind == ABILU_ORDER_RCM) {
        std::vector<int> mask(n, 0);
        rcm(g, mask, 0, level, out);
    } else if (kind == ABILU_ORDER_1WD) {
        std::vector<int> mask(n, 0);
        one_way(g, mask, 0, level, out);
    } else {
        std::vector<double> w((size_t)nnzb);
        for (int64_t p = 0; p < nnzb; p++) {
            if (weights) {
                w[p] = weights[p];
            } else {
                double s = 0.0;
                for (int k = 0; k < BB; k++) s += vals[p * BB + k] * vals[p * BB + k];
                w[p] = sqrt(s);
            }
        }
        std::vector<std::vector<int>> lines;
        find_lines(g, rowptr, colind, w.data(), line_threshold, line_of, lines);
        const int nl = (int)lines.size();
        // quotient graph: vertex k < nl = line k, nl + c = cell c in no line
        std::vector<int> vid(n), cell_of_v;
        int nv = nl;
        for (int c = 0; c < n; c++) {
            if (line_of[c] >= 0) vid[c] = line_of[c];
            else { vid[c] = nv++; cell_of_v.push_back(c); }
        }
        std::vector<int> vorder;
        if (kind == ABILU_ORDER_LINE) {  // position of each vertex's first cell
            std::vector<char> seen(nv, 0);
            for (int c = 0; c < n; c++)
                if (!seen[vid[c]]) { seen[vid[c]] = 1; vorder.push_back(vid[c]); }
        } else {
            std::vector<std::pair<int, int>> e;
            for (int i = 0; i < n; i++)
                for (int p = g.ptr[i]; p < g.ptr[i + 1]; p++)
                    if (vid[i] != vid[g.adj[p]]) e.emplace_back(vid[i], vid[g.adj[p]]);
            std::sort(e.begin(), e.end());
            e.erase(std::unique(e.begin(), e.end()), e.end());
            Graph q;
            q.n = nv;
            q.ptr.assign(nv + 1, 0);
            for (auto &x : e) q.ptr[x.first + 1]++;
            for (int v = 0; v < nv; v++) q.ptr[v + 1] += q.ptr[v];
            q.adj.resize(e.size());
            for (size_t k = 0; k < e.size(); k++) q.adj[k] = e[k].second;
            std::vector<int> qlevel(nv, -1), qmask(nv, 0);
            if (kind == ABILU_ORDER_LINE_RCM) rcm(q, qmask, 0, qlevel, vorder);
            else one_way(q, qmask, 0, qlevel, vorder);
        }
        for (int v : vorder) {
            if (v < nl) out.insert(out.end(), lines[v].begin(), lines[v].end());
            else out.push_back(cell_of_v[v - nl]);
        }
    }
    if ((int)out.size() != n) return fail(ABILU_EINVAL, "order: internal error (%zu of %d cells)", out.size(), n);
    for (int k = 0; k < n; k++) perm[k] = out[k];
    if (line_of_out)
        for (int c = 0; c < n; c++) line_of_out[c] = line_of[c];
    return ABILU_OK;
}

extern "C" abilu_status abilu_permute_pattern(int32_t n, const int32_t *rowptr, const int32_t *colind,
                                              const int32_t *perm, int32_t *rowptr_out,
                                              int32_t *colind_out, int32_t *src_out) {
    if (n < 1 || !rowptr || !colind || !perm || !rowptr_out || !colind_out || !src_out)
        return fail(ABILU_EINVAL, "permute_pattern: NULL argument");
    std::vector<int> inv(n, -1);
    for (int k = 0; k < n; k++) {
        if (perm[k] < 0 || perm[k] >= n || inv[perm[k]] >= 0)
            return fail(ABILU_EINVAL, "permute_pattern: perm is not a permutation");
        inv[perm[k]] = k;
    }
    rowptr_out[0] = 0;
    std::vector<std::pair<int, int>> row;
    for (int k = 0; k < n; k++) {
        const int i = perm[k];
        row.clear();
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) row.emplace_back(inv[colind[p]], p);
        std::sort(row.begin(), row.end());
        int o = rowptr_out[k];
        for (auto &x : row) {
            colind_out[o] = x.first;
            src_out[o] = x.second;
            o++;
        }
        rowptr_out[k + 1] = o;
    }
    return ABILU_OK;
}

namespace abilu {
__global__ void k_gather_blocks(long long nnzb, const int32_t *__restrict__ src,
                                const double *__restrict__ in, double *__restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // (block, row q)
    if (e >= nnzb * 4) return;
    const long long p = e >> 2;
    const int q = (int)(e & 3);
    double v[4];
    ld_row(in + (size_t)src[p] * BB + q * BS, v);
    st_row(out + (size_t)p * BB + q * BS, v);
}
}  // namespace abilu

extern "C" abilu_status abilu_gather_blocks(int64_t nnzb, const int32_t *src, const double *vals_in,
                                            double *vals_out, abilu_stream stream) {
    if (nnzb < 0 || (nnzb > 0 && (!src || !vals_in || !vals_out)))
        return fail(ABILU_EINVAL, "gather_blocks: bad argument");
    if (vals_in == vals_out) return fail(ABILU_EINVAL, "gather_blocks: in and out must differ");
    if (nnzb == 0) return ABILU_OK;
    k_gather_blocks<<<counted((int)((nnzb * 4 + 255) / 256)), 256, 0, S(stream)>>>(nnzb, src, vals_in,
                                                                               vals_out);
    ABILU_LAUNCH_CHECK("k_gather_blocks");
    return ABILU_OK;
}
