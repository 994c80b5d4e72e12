/*
 * Orderings of the cell graph (Sec. 5: reverse Cuthill-McKee and one-way
 * dissection; Sec. 5.1: lines of strongly coupled cells; Sec. 5.2: the hybrid
 * line-RCM and line-1WD orderings) -- oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain single-threaded C written from the rules
 * below; it shares no code with the CUDA library, and only the test suite
 * loads it.  The paper names the orderings (it used PETSc's RCM and a one-way
 * dissection for unstructured grids, and Mavriplis's line detection) without
 * their tie-breaks; the rules here are this project's readings of them, the
 * same ones the library documents for abilu_order.
 *
 * Graph.  Cells i != j are adjacent when block (i,j) or (j,i) is in the
 *   pattern; neighbour lists ascend; the degree of a cell is its number of
 *   neighbours in the whole graph (also when a subset of it is ordered).
 * Level structure from r over a cell set: breadth first, each cell's
 *   neighbours taken in ascending index.
 * Pseudo-peripheral cell of a connected set, searched from s: r = s; x = the
 *   cell of least degree in the last level of r's level structure (ties: the
 *   lowest index); if x's level structure has more levels than r's, r = x and
 *   repeat; otherwise the answer is r.
 * Cuthill-McKee from r: a queue starting with r; each cell taken from the
 *   queue appends its neighbours in the set that are not yet numbered, in
 *   increasing (degree, index).  Reverse Cuthill-McKee (RCM) is that order
 *   reversed.
 * RCM of a cell set: its connected components in order of their lowest cell,
 *   each numbered by RCM from the pseudo-peripheral cell searched from that
 *   lowest cell.
 * One-way dissection (1WD), George's spacing: per component (lowest cell
 *   first), the level structure from its pseudo-peripheral cell has L levels;
 *   w = cells / L, delta = max(2, round(sqrt((3 w + 13) / 2))) (halves away
 *   from zero).  If L < 2 delta + 1 the component is numbered by RCM.
 *   Otherwise the levels delta, 2 delta, ... below L - 1 are separators; the
 *   rest of the component splits into blocks (connected pieces), taken in the
 *   order of their first cell in the level structure's breadth-first order and
 *   each numbered by RCM with the pseudo-peripheral search from that cell.  The
 *   separator cells of all components come last, component by component, in
 *   breadth-first order.
 * Lines (Sec. 5.1).  Block weight: the caller's, or the Frobenius norm of the
 *   block (squares summed in storage order).  Coupling w(i,j) of an edge: the
 *   larger weight of blocks (i,j) and (j,i).  wmax_i, wmin_i: the largest and
 *   smallest coupling of cell i (0 with no neighbour); anisotropy a_i =
 *   wmax_i / wmin_i (infinite when wmin_i = 0 < wmax_i, 1 when wmax_i = 0).  A
 *   cell is anisotropic when a_i >= tau.  Seeds: cells by decreasing a_i (ties:
 *   ascending index), up to the first that is not anisotropic.  A seed in no
 *   line starts one; the line grows from the seed forward, then backward:
 *   from its end c, the free neighbour u (in no line) with the largest w(c,u)
 *   (ties: lowest index) joins when w(c,u) >= tau rho and tau w(c,u) >=
 *   wmax_u, where rho = wmin_c for an anisotropic c and otherwise the wmin of
 *   the last anisotropic cell of the line, and when u is anisotropic or fewer
 *   than two cells without anisotropy end the line (at most two such cells in
 *   a row).  A line of one cell is dropped (the seed stays free).  A line's
 *   cells run from the backward end through the seed to the forward end; lines
 *   are numbered by their lowest cell.
 * LINE: lines and free cells in the order of their first cell in the input
 *   numbering, each line contiguous.  LINE_RCM / LINE_1WD: the graph whose
 *   vertices are the lines (numbered 0..nl-1) and the free cells (nl, nl+1,
 *   ... in ascending cell index), two vertices adjacent when any of their
 *   cells are, ordered by RCM / 1WD with the rules above, each line expanded
 *   in place.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int32_t idx_t;

typedef struct {
    idx_t n;
    idx_t *ptr;   /* n + 1 */
    idx_t *nb;    /* ptr[n] neighbours, ascending per cell */
} graph;

static int cmp_idx(const void *a, const void *b)
{
    idx_t x = *(const idx_t *)a, y = *(const idx_t *)b;
    return (x > y) - (x < y);
}

/* graph from m directed pairs (u[k], v[k]) (both directions are added, self
 * pairs ignored, duplicates removed) */
static int make_graph(idx_t n, long m, const idx_t *u, const idx_t *v, graph *g)
{
    idx_t *cnt = calloc((size_t)n + 1, sizeof(idx_t));
    if (!cnt) return -1;
    for (long k = 0; k < m; k++)
        if (u[k] != v[k]) { cnt[u[k] + 1]++; cnt[v[k] + 1]++; }
    for (idx_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    idx_t *fill = malloc(sizeof(idx_t) * ((size_t)n + 1));
    idx_t *nb = malloc(sizeof(idx_t) * ((size_t)cnt[n] + 1));
    if (!fill || !nb) { free(cnt); free(fill); free(nb); return -1; }
    memcpy(fill, cnt, sizeof(idx_t) * ((size_t)n + 1));
    for (long k = 0; k < m; k++)
        if (u[k] != v[k]) { nb[fill[u[k]]++] = v[k]; nb[fill[v[k]]++] = u[k]; }
    /* sort each list and squeeze out repeats */
    idx_t w = 0;
    for (idx_t i = 0; i < n; i++) {
        idx_t b = cnt[i], e = cnt[i + 1];
        qsort(nb + b, (size_t)(e - b), sizeof(idx_t), cmp_idx);
        cnt[i] = w;
        for (idx_t p = b; p < e; p++)
            if (p == b || nb[p] != nb[p - 1]) nb[w++] = nb[p];
    }
    cnt[n] = w;
    free(fill);
    g->n = n;
    g->ptr = cnt;
    g->nb = nb;
    return 0;
}

static void free_graph(graph *g)
{
    free(g->ptr);
    free(g->nb);
}

static idx_t deg(const graph *g, idx_t v) { return g->ptr[v + 1] - g->ptr[v]; }

/* Breadth-first level structure from r over the cells with set[c] == tag.
 * lev[] must be -1 on those cells; it is filled for the cells reached, whose
 * breadth-first order goes to seq[]; returns their number, *nlev the number of
 * levels.  The caller resets lev[] (reset_levels). */
static idx_t levels_from(const graph *g, idx_t r, const idx_t *set, idx_t tag, idx_t *lev,
                         idx_t *seq, idx_t *nlev)
{
    idx_t head = 0, tail = 0;
    seq[tail++] = r;
    lev[r] = 0;
    while (head < tail) {
        idx_t v = seq[head++];
        for (idx_t p = g->ptr[v]; p < g->ptr[v + 1]; p++) {
            idx_t u = g->nb[p];
            if (set[u] == tag && lev[u] < 0) {
                lev[u] = lev[v] + 1;
                seq[tail++] = u;
            }
        }
    }
    *nlev = lev[seq[tail - 1]] + 1;
    return tail;
}

static void reset_levels(idx_t *lev, const idx_t *seq, idx_t k)
{
    for (idx_t t = 0; t < k; t++) lev[seq[t]] = -1;
}

static idx_t pseudo_peripheral(const graph *g, idx_t s, const idx_t *set, idx_t tag, idx_t *lev,
                               idx_t *seq)
{
    idx_t r = s, depth_r;
    idx_t k = levels_from(g, r, set, tag, lev, seq, &depth_r);
    for (;;) {
        idx_t x = -1;
        for (idx_t t = 0; t < k; t++) {
            idx_t v = seq[t];
            if (lev[v] != depth_r - 1) continue;
            if (x < 0 || deg(g, v) < deg(g, x) || (deg(g, v) == deg(g, x) && v < x)) x = v;
        }
        reset_levels(lev, seq, k);
        idx_t depth_x;
        k = levels_from(g, x, set, tag, lev, seq, &depth_x);
        if (depth_x > depth_r) {
            r = x;
            depth_r = depth_x;
            continue;
        }
        reset_levels(lev, seq, k);
        /* the last search was x's; r's structure is not needed further */
        return r;
    }
}

/* key of the Cuthill-McKee neighbour order */
static const graph *cm_graph;
static int cmp_deg_idx(const void *a, const void *b)
{
    idx_t x = *(const idx_t *)a, y = *(const idx_t *)b;
    idx_t dx = deg(cm_graph, x), dy = deg(cm_graph, y);
    if (dx != dy) return dx < dy ? -1 : 1;
    return (x > y) - (x < y);
}

/* Cuthill-McKee numbering from r of the cells with set[c] == tag reachable
 * from it, written to out[]; numbered[] marks them.  Returns the count. */
static idx_t cuthill_mckee(const graph *g, idx_t r, const idx_t *set, idx_t tag, char *numbered,
                           idx_t *out)
{
    idx_t head = 0, tail = 0;
    out[tail++] = r;
    numbered[r] = 1;
    cm_graph = g;
    while (head < tail) {
        idx_t v = out[head++];
        idx_t first = tail;
        for (idx_t p = g->ptr[v]; p < g->ptr[v + 1]; p++) {
            idx_t u = g->nb[p];
            if (set[u] == tag && !numbered[u]) {
                numbered[u] = 1;
                out[tail++] = u;
            }
        }
        qsort(out + first, (size_t)(tail - first), sizeof(idx_t), cmp_deg_idx);
    }
    return tail;
}

static void reverse(idx_t *a, idx_t k)
{
    for (idx_t i = 0, j = k - 1; i < j; i++, j--) {
        idx_t t = a[i];
        a[i] = a[j];
        a[j] = t;
    }
}

/* RCM of the connected cells of set == tag reached from s, appended at out */
static idx_t rcm_piece(const graph *g, idx_t s, const idx_t *set, idx_t tag, char *numbered,
                       idx_t *lev, idx_t *seq, idx_t *out)
{
    idx_t r = pseudo_peripheral(g, s, set, tag, lev, seq);
    idx_t k = cuthill_mckee(g, r, set, tag, numbered, out);
    reverse(out, k);
    return k;
}

/* RCM of every component of the whole graph (set all zero); returns count */
static idx_t rcm_all(const graph *g, idx_t *out)
{
    idx_t n = g->n, k = 0;
    idx_t *set = calloc((size_t)n, sizeof(idx_t));
    idx_t *lev = malloc(sizeof(idx_t) * (size_t)n);
    idx_t *seq = malloc(sizeof(idx_t) * (size_t)n);
    char *numbered = calloc((size_t)n, 1);
    for (idx_t i = 0; i < n; i++) lev[i] = -1;
    for (idx_t s = 0; s < n; s++)
        if (!numbered[s]) k += rcm_piece(g, s, set, 0, numbered, lev, seq, out + k);
    free(set); free(lev); free(seq); free(numbered);
    return k;
}

/* one-way dissection of the whole graph; returns count */
static idx_t onewd_all(const graph *g, idx_t *out)
{
    idx_t n = g->n, k = 0, nsep = 0;
    idx_t *set = calloc((size_t)n, sizeof(idx_t));   /* 0: ordinary, 1: separator */
    idx_t *lev = malloc(sizeof(idx_t) * (size_t)n);
    idx_t *seq = malloc(sizeof(idx_t) * (size_t)n);
    idx_t *comp = malloc(sizeof(idx_t) * (size_t)n);
    idx_t *clev = malloc(sizeof(idx_t) * (size_t)n);
    idx_t *seps = malloc(sizeof(idx_t) * (size_t)n);
    char *numbered = calloc((size_t)n, 1);
    char *done = calloc((size_t)n, 1);
    for (idx_t i = 0; i < n; i++) lev[i] = -1;
    for (idx_t s = 0; s < n; s++) {
        if (done[s]) continue;
        idx_t r = pseudo_peripheral(g, s, set, 0, lev, seq);
        idx_t L;
        idx_t size = levels_from(g, r, set, 0, lev, comp, &L);
        for (idx_t t = 0; t < size; t++) {
            clev[t] = lev[comp[t]];
            done[comp[t]] = 1;
        }
        reset_levels(lev, comp, size);
        double w = (double)size / (double)L;
        long delta = lround(sqrt((3.0 * w + 13.0) / 2.0));
        if (delta < 2) delta = 2;
        if (L < 2 * delta + 1) {
            k += rcm_piece(g, s, set, 0, numbered, lev, seq, out + k);
            continue;
        }
        for (idx_t t = 0; t < size; t++) {
            idx_t l = clev[t];
            if (l > 0 && l % delta == 0 && l < L - 1) {
                set[comp[t]] = 1;
                seps[nsep++] = comp[t];
            }
        }
        for (idx_t t = 0; t < size; t++) {
            idx_t v = comp[t];
            if (set[v] == 0 && !numbered[v])
                k += rcm_piece(g, v, set, 0, numbered, lev, seq, out + k);
        }
    }
    memcpy(out + k, seps, sizeof(idx_t) * (size_t)nsep);
    k += nsep;
    free(set); free(lev); free(seq); free(comp); free(clev); free(seps);
    free(numbered); free(done);
    return k;
}

/* seeds: decreasing anisotropy, then ascending index */
static const double *seed_key;
static int cmp_seed(const void *a, const void *b)
{
    idx_t x = *(const idx_t *)a, y = *(const idx_t *)b;
    if (seed_key[x] != seed_key[y]) return seed_key[x] > seed_key[y] ? -1 : 1;
    return (x > y) - (x < y);
}

static idx_t slot_of(const graph *g, idx_t i, idx_t j)
{
    idx_t lo = g->ptr[i], hi = g->ptr[i + 1];
    while (lo < hi) {
        idx_t mid = lo + (hi - lo) / 2;
        if (g->nb[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return (lo < g->ptr[i + 1] && g->nb[lo] == j) ? lo : -1;
}

/* Lines of strongly coupled cells.  line_of[c] = line index or -1; the cells
 * of line l are lcell[lstart[l] .. lstart[l+1]).  Returns the line count. */
static idx_t find_lines(const graph *g, const idx_t *rowptr, const idx_t *colind,
                        const double *wblk, double tau, idx_t *line_of, idx_t *lcell,
                        idx_t *lstart)
{
    idx_t n = g->n;
    double *wadj = calloc((size_t)g->ptr[n] + 1, sizeof(double));
    double *wmax = malloc(sizeof(double) * (size_t)n), *wmin = malloc(sizeof(double) * (size_t)n);
    double *an = malloc(sizeof(double) * (size_t)n);
    idx_t *seeds = malloc(sizeof(idx_t) * (size_t)n);
    idx_t *fwd = malloc(sizeof(idx_t) * (size_t)n), *bwd = malloc(sizeof(idx_t) * (size_t)n);
    idx_t *tmp_cell = malloc(sizeof(idx_t) * (size_t)n), *tmp_start = malloc(sizeof(idx_t) * ((size_t)n + 1));
    for (idx_t i = 0; i < n; i++)
        for (idx_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            if (j == i) continue;
            idx_t a = slot_of(g, i, j), b = slot_of(g, j, i);
            if (wblk[p] > wadj[a]) wadj[a] = wblk[p];
            if (wblk[p] > wadj[b]) wadj[b] = wblk[p];
        }
    for (idx_t i = 0; i < n; i++) {
        double hi = 0.0, lo = 0.0;
        for (idx_t p = g->ptr[i]; p < g->ptr[i + 1]; p++) {
            if (p == g->ptr[i] || wadj[p] > hi) hi = wadj[p];
            if (p == g->ptr[i] || wadj[p] < lo) lo = wadj[p];
        }
        wmax[i] = hi;
        wmin[i] = lo;
        if (hi == 0.0) an[i] = 1.0;
        else if (lo == 0.0) an[i] = INFINITY;
        else an[i] = hi / lo;
        seeds[i] = i;
        line_of[i] = -1;
    }
    seed_key = an;
    qsort(seeds, (size_t)n, sizeof(idx_t), cmp_seed);
    idx_t nlines = 0, ncell = 0;
    tmp_start[0] = 0;
    for (idx_t t = 0; t < n; t++) {
        idx_t s = seeds[t];
        if (an[s] < tau) break;
        if (line_of[s] >= 0) continue;
        line_of[s] = nlines;
        idx_t nf = 0, nbk = 0;
        for (int dir = 0; dir < 2; dir++) {   /* forward, then backward */
            idx_t *part = dir == 0 ? fwd : bwd;
            idx_t *np = dir == 0 ? &nf : &nbk;
            double ref = wmin[s];
            int run = 0;
            idx_t c = s;
            for (;;) {
                idx_t best = -1;
                double bw = 0.0;
                for (idx_t p = g->ptr[c]; p < g->ptr[c + 1]; p++) {
                    idx_t u = g->nb[p];
                    if (line_of[u] >= 0) continue;
                    if (best < 0 || wadj[p] > bw) { best = u; bw = wadj[p]; }
                }
                if (best < 0) break;
                double rho = an[c] >= tau ? wmin[c] : ref;
                if (bw < tau * rho || tau * bw < wmax[best]) break;
                int plain = an[best] < tau;
                if (plain && run == 2) break;
                line_of[best] = nlines;
                part[(*np)++] = best;
                if (plain) run++;
                else { run = 0; ref = wmin[best]; }
                c = best;
            }
        }
        if (nf + nbk == 0) {   /* a single cell is not a line */
            line_of[s] = -1;
            continue;
        }
        for (idx_t q = nbk - 1; q >= 0; q--) tmp_cell[ncell++] = bwd[q];
        tmp_cell[ncell++] = s;
        for (idx_t q = 0; q < nf; q++) tmp_cell[ncell++] = fwd[q];
        tmp_start[++nlines] = ncell;
    }
    /* number the lines by their lowest cell: scan cells in ascending order */
    idx_t *newid = malloc(sizeof(idx_t) * ((size_t)nlines + 1));
    for (idx_t l = 0; l < nlines; l++) newid[l] = -1;
    idx_t next = 0, at = 0;
    lstart[0] = 0;
    for (idx_t c = 0; c < n; c++) {
        idx_t l = line_of[c];
        if (l < 0 || newid[l] >= 0) continue;
        newid[l] = next++;
        for (idx_t q = tmp_start[l]; q < tmp_start[l + 1]; q++) lcell[at++] = tmp_cell[q];
        lstart[next] = at;
    }
    for (idx_t c = 0; c < n; c++)
        if (line_of[c] >= 0) line_of[c] = newid[line_of[c]];
    free(newid); free(wadj); free(wmax); free(wmin); free(an); free(seeds); free(fwd); free(bwd);
    free(tmp_cell); free(tmp_start);
    return nlines;
}

/*
 * orc_order: perm[k] = the old index of the cell numbered k; line_of (may be
 * NULL) = each cell's line or -1.  kind: 0 RCM, 1 1WD, 2 LINE, 3 LINE_RCM,
 * 4 LINE_1WD.  weights (per block) or vals (4x4 blocks) give the couplings of
 * the line kinds.  Returns 0, or -1 on bad input.
 */
int orc_order(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *weights,
              const double *vals, int kind, double tau, idx_t *perm, idx_t *line_of_out)
{
    if (n < 1 || kind < 0 || kind > 4) return -1;
    long nnzb = rowptr[n];
    idx_t *rows = malloc(sizeof(idx_t) * ((size_t)nnzb + 1));
    for (idx_t i = 0; i < n; i++)
        for (idx_t p = rowptr[i]; p < rowptr[i + 1]; p++) rows[p] = i;
    graph g;
    if (make_graph(n, nnzb, rows, colind, &g)) { free(rows); return -1; }
    idx_t *line_of = malloc(sizeof(idx_t) * (size_t)n);
    for (idx_t i = 0; i < n; i++) line_of[i] = -1;
    int rc = 0;
    if (kind == 0) {
        rcm_all(&g, perm);
    } else if (kind == 1) {
        onewd_all(&g, perm);
    } else {
        if (!weights && !vals) { rc = -1; goto out; }
        double *w = malloc(sizeof(double) * ((size_t)nnzb + 1));
        for (long p = 0; p < nnzb; p++) {
            if (weights) {
                w[p] = weights[p];
            } else {
                double s = 0.0;
                for (int e = 0; e < 16; e++) s += vals[p * 16 + e] * vals[p * 16 + e];
                w[p] = sqrt(s);
            }
        }
        idx_t *lcell = malloc(sizeof(idx_t) * (size_t)n);
        idx_t *lstart = malloc(sizeof(idx_t) * ((size_t)n + 1));
        idx_t nl = find_lines(&g, rowptr, colind, w, tau, line_of, lcell, lstart);
        free(w);
        /* vertex of each cell: its line, or nl + rank among free cells */
        idx_t *vid = malloc(sizeof(idx_t) * (size_t)n);
        idx_t *vcell = malloc(sizeof(idx_t) * (size_t)n);   /* free vertex -> cell */
        idx_t nv = nl;
        for (idx_t c = 0; c < n; c++) {
            if (line_of[c] >= 0) vid[c] = line_of[c];
            else { vcell[nv - nl] = c; vid[c] = nv++; }
        }
        idx_t *vord = malloc(sizeof(idx_t) * (size_t)nv);
        if (kind == 2) {
            char *seen = calloc((size_t)nv, 1);
            idx_t k = 0;
            for (idx_t c = 0; c < n; c++)
                if (!seen[vid[c]]) { seen[vid[c]] = 1; vord[k++] = vid[c]; }
            free(seen);
        } else {
            idx_t *qu = malloc(sizeof(idx_t) * ((size_t)g.ptr[n] + 1));
            idx_t *qv = malloc(sizeof(idx_t) * ((size_t)g.ptr[n] + 1));
            long m = 0;
            for (idx_t i = 0; i < n; i++)
                for (idx_t p = g.ptr[i]; p < g.ptr[i + 1]; p++)
                    if (vid[i] != vid[g.nb[p]]) { qu[m] = vid[i]; qv[m] = vid[g.nb[p]]; m++; }
            graph q;
            make_graph(nv, m, qu, qv, &q);
            free(qu); free(qv);
            if (kind == 3) rcm_all(&q, vord);
            else onewd_all(&q, vord);
            free_graph(&q);
        }
        idx_t k = 0;
        for (idx_t t = 0; t < nv; t++) {
            idx_t v = vord[t];
            if (v < nl)
                for (idx_t q = lstart[v]; q < lstart[v + 1]; q++) perm[k++] = lcell[q];
            else
                perm[k++] = vcell[v - nl];
        }
        free(vid); free(vcell); free(vord); free(lcell); free(lstart);
    }
    if (line_of_out)
        for (idx_t i = 0; i < n; i++) line_of_out[i] = line_of[i];
out:
    free(rows);
    free(line_of);
    free_graph(&g);
    return rc;
}
