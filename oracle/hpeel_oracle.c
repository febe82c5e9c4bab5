/*
 * hpeel_oracle.c -- CPU oracle for hypergraph peeling and MWHC minimal
 * perfect hashing ("Cache-Oblivious Peeling of Random Hypergraphs",
 * Belazzougui, Boldi, Ottaviano, Venturini, Vigna).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, table or constant generator with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Every function states the definition it follows; there is no blocking,
 * fusion or reordering beyond what that definition states.
 *
 * Readings of the paper taken here (the paper is silent on these points):
 *  - vertex count: m = r * ceil(ceil(gamma_milli * n / 1000) / r), integer
 *    arithmetic, so part size P = m / r (sec. 4.3, tripartition);
 *  - hash: vertex j of key k is (mix64(k ^ (seed + j)) mod P) + j * P, where
 *    mix64 is the SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014);
 *    the paper uses a Jenkins hash (sec. 3, footnote) -- any fixed seeded
 *    hash defines the same problem relative to its edge list;
 *  - hinge: when several vertices of an edge have degree 1 in the round the
 *    edge is peeled, the hinge (the index i of sec. 3's MPHF construction)
 *    is the one of smallest position j;
 *  - canonical order: layers in round order, ascending edge id inside a
 *    layer (sec. 4.2 leaves the intra-layer order free), unpeeled (core)
 *    edges last in ascending id;
 *  - g encoding: 2 bits per vertex; an assigned value 0 is stored as 3 so
 *    that "assigned" is "non-zero" for the rank structure; unassigned = 0;
 *  - rank directory: one cumulative 64-bit count per 512 vertices;
 *  - general (not r-partite) hypergraphs: vertices in [0, m) in any
 *    position, a row may repeat a vertex and degrees count occurrences (a
 *    vertex of degree 1 then occurs once in its only edge); the position of
 *    a degree-1 vertex in its edge is read off the edge's row, and the hinge
 *    is again the smallest such position;
 *  - static functions (sec. 3, f: S -> [sigma]): 2 <= sigma <= 2^32,
 *    b = ceil(log2 sigma) bits per vertex, u[v] at bits [v b, (v + 1) b) of
 *    one bit string (bit i = bit i mod 64 of word i / 64), values stored as
 *    they are (no "0 as 3" code: a static function needs no rank), vertices
 *    never a hinge hold 0, a value >= sigma is an input error.
 *
 * Parity status: every function here is pinned by tests against closed
 * forms, published test vectors, brute force or independent invariants.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_UNCLAIMED 0xFFFFFFFFu
#define ORC_MAX_R 4

/* Error codes returned by the oracle. */
#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EINTERNAL 3
#define ORC_ELAYERS 4 /* layer_off too small for the number of rounds */
#define ORC_ERETRIES 5

/* ---------------------------------------------------------------------- */
/* Hashing (sec. 3, sec. 4.3 "Exploiting the tripartition").              */
/* ---------------------------------------------------------------------- */

/* SplitMix64 output function ("mix64"): two xorshift-multiply steps and a
 * final xorshift, all modulo 2^64 (Steele, Lea, Flood 2014). */
uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Number of vertices for n edges at sparsity gamma = gamma_milli / 1000,
 * rounded up to a multiple of r so the r parts have equal size. */
uint64_t orc_num_vertices(uint64_t n, uint32_t gamma_milli, uint32_t r)
{
    uint64_t gn = (gamma_milli * n + 999u) / 1000u; /* ceil(gamma n) */
    uint64_t parts = (gn + r - 1) / r;
    return parts * r;
}

/* Edge of key i: vertex j lies in part j, i.e. in [j P, (j + 1) P)
 * (sec. 4.3: h_j has codomain [j |V| / r, (j + 1) |V| / r)). */
int orc_hash_edges(const uint64_t *keys, uint64_t n, uint64_t m, uint32_t r,
                   uint64_t seed, uint32_t *edges)
{
    if (r < 2 || r > ORC_MAX_R || m % r != 0 || m >= (1ull << 32))
        return ORC_EINVAL;
    if (n == 0)
        return ORC_OK;
    if (m == 0)
        return ORC_EINVAL;
    uint64_t P = m / r;
    for (uint64_t i = 0; i < n; i++)
        for (uint32_t j = 0; j < r; j++) {
            uint64_t h = orc_mix64(keys[i] ^ (seed + j));
            edges[i * r + j] = (uint32_t)(h % P + (uint64_t)j * P);
        }
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Packed incidence lists, XOR trick (sec. 4.1).                         */
/* ---------------------------------------------------------------------- */

/* deg[v] = number of edges containing v; x[v] = XOR of the ids of those
 * edges (the labelled form of the packed incidence list, where the label of
 * an edge is its id).  When deg[v] == 1, x[v] is the id of v's only edge. */
int orc_incidence(const uint32_t *edges, uint64_t n, uint64_t m, uint32_t r,
                  uint32_t *deg, uint32_t *x)
{
    if (r < 2 || r > ORC_MAX_R)
        return ORC_EINVAL;
    memset(deg, 0, m * sizeof(uint32_t));
    memset(x, 0, m * sizeof(uint32_t));
    for (uint64_t e = 0; e < n; e++)
        for (uint32_t j = 0; j < r; j++) {
            uint32_t v = edges[e * r + j];
            if (v >= m)
                return ORC_EINVAL;
            deg[v] += 1;
            x[v] ^= (uint32_t)e;
        }
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Layered (round-synchronous) peeling (sec. 4.2).                       */
/* ---------------------------------------------------------------------- */

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

/* Round-synchronous peel.
 *
 * Round t: F_t is the set of vertices of degree 1 in the graph left after
 * rounds 0..t-1.  Every edge retrieved from a vertex of F_t (the only edge
 * of that vertex, read off the packed incidence list) forms layer L_t; an
 * edge reached from several vertices of F_t enters L_t once (the paper's
 * deduplication of D_i into P_i).  Then every edge of L_t is deleted from
 * the incidence lists of all its vertices (DeleteEdge), and F_{t+1} is the
 * set of vertices of degree 1 afterwards.  Vertices that reach degree 1 in
 * round t were touched by that round's deletions, and every vertex of F_t
 * falls to degree 0 in round t, so F_{t+1} is taken from the touched
 * vertices only; that restricts the scan and changes no result.
 *
 * Outputs:
 *  order[n]         canonical order: L_0 ascending, L_1 ascending, ...,
 *                   then the unpeeled (2-core) edges ascending;
 *  claim[n]         (t << 2) | hinge for an edge peeled in round t, where
 *                   hinge is the smallest position j whose vertex was in
 *                   F_t; ORC_UNCLAIMED for core edges;
 *  layer_off[R+1]   start of L_t in order, layer_off[R] = number peeled
 *                   (capacity max_layers + 1 entries; may be NULL);
 *  *rounds          R, the number of non-empty layers;
 *  *n_peeled        |L_0| + ... + |L_{R-1}|.
 */
/* Position of vertex v in the row of edge e: the first j with row[j] == v
 * (a vertex of degree 1 occurs once in its only edge). */
static uint32_t row_position(const uint32_t *edges, uint64_t e, uint32_t r, uint32_t v)
{
    for (uint32_t j = 0; j < r; j++)
        if (edges[e * r + j] == v)
            return j;
    return r;
}

/* general = 0: r-partite graph, the position of v is its part v / P
 * (sec. 4.3); general = 1: any r-hypergraph on [0, m) (sec. 2: edges are
 * r-subsets; rows may repeat a vertex, degrees count occurrences), the
 * position of v in an edge is read off the edge's row. */
static int peel_rounds_impl(const uint32_t *edges, uint64_t n, uint64_t m, uint32_t r,
                            uint32_t *order, uint32_t *claim, uint64_t *layer_off,
                            uint64_t max_layers, uint32_t *rounds, uint64_t *n_peeled,
                            int general)
{
    /* n = 0 is the empty graph, whatever m (an empty bucket has m = 0) */
    if (r < 2 || r > ORC_MAX_R || n >= (1ull << 32) || (n > 0 && m == 0) ||
        (!general && (m % r) != 0))
        return ORC_EINVAL;
    *rounds = 0;
    *n_peeled = 0;
    if (n == 0) {
        if (layer_off)
            layer_off[0] = 0;
        return ORC_OK;
    }
    uint64_t P = m / r;
    int rc = ORC_OK;
    uint32_t *deg = malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t *x = malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t *F = malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t *T = malloc((n * r) * sizeof(uint32_t));
    uint32_t *L = malloc(n * sizeof(uint32_t));
    if (!deg || !x || !F || !T || !L) {
        rc = ORC_ENOMEM;
        goto out;
    }
    rc = orc_incidence(edges, n, m, r, deg, x);
    if (rc)
        goto out;
    for (uint64_t e = 0; e < n; e++)
        claim[e] = ORC_UNCLAIMED;

    uint64_t nF = 0;
    for (uint64_t v = 0; v < m; v++)
        if (deg[v] == 1)
            F[nF++] = (uint32_t)v;

    uint64_t peeled = 0;
    uint32_t t = 0;
    while (nF > 0) {
        if (t >= (1u << 30) - 1) {
            rc = ORC_EINTERNAL;
            goto out;
        }
        /* (i) retrieve, all against the same snapshot of the lists. */
        uint64_t nL = 0;
        for (uint64_t k = 0; k < nF; k++) {
            uint32_t v = F[k];
            if (deg[v] != 1) { /* cannot happen: F holds degree-1 vertices */
                rc = ORC_EINTERNAL;
                goto out;
            }
            uint32_t e = x[v];
            uint32_t j = general ? row_position(edges, e, r, v) : (uint32_t)(v / P);
            if (j >= r) { /* cannot happen: v is a vertex of its only edge */
                rc = ORC_EINTERNAL;
                goto out;
            }
            uint32_t tag = (t << 2) | j;
            if (claim[e] == ORC_UNCLAIMED) {
                claim[e] = tag;
                L[nL++] = e;
            } else if ((claim[e] >> 2) == t) {
                if (tag < claim[e])
                    claim[e] = tag; /* smallest position wins the hinge */
            } else { /* an edge of an earlier layer cannot be retrieved */
                rc = ORC_EINTERNAL;
                goto out;
            }
        }
        /* (ii) the layer, ascending edge id. */
        qsort(L, nL, sizeof(uint32_t), cmp_u32);
        if (layer_off) {
            if (t >= max_layers) {
                rc = ORC_ELAYERS;
                goto out;
            }
            layer_off[t] = peeled;
        }
        for (uint64_t k = 0; k < nL; k++)
            order[peeled + k] = L[k];
        peeled += nL;
        /* (iii) DeleteEdge on every vertex of every edge of the layer. */
        uint64_t nT = 0;
        for (uint64_t k = 0; k < nL; k++) {
            uint32_t e = L[k];
            for (uint32_t j = 0; j < r; j++) {
                uint32_t w = edges[(uint64_t)e * r + j];
                deg[w] -= 1;
                x[w] ^= e;
                T[nT++] = w;
            }
        }
        /* (iv) next frontier: touched vertices now of degree 1. */
        qsort(T, nT, sizeof(uint32_t), cmp_u32);
        nF = 0;
        for (uint64_t k = 0; k < nT; k++) {
            if (k > 0 && T[k] == T[k - 1])
                continue;
            if (deg[T[k]] == 1)
                F[nF++] = T[k];
        }
        t += 1;
    }
    /* core edges, ascending, after the layers */
    uint64_t pos = peeled;
    for (uint64_t e = 0; e < n; e++)
        if (claim[e] == ORC_UNCLAIMED)
            order[pos++] = (uint32_t)e;
    if (layer_off) {
        if (t > max_layers) {
            rc = ORC_ELAYERS;
            goto out;
        }
        layer_off[t] = peeled;
    }
    *rounds = t;
    *n_peeled = peeled;
out:
    free(deg);
    free(x);
    free(F);
    free(T);
    free(L);
    return rc;
}

int orc_peel_rounds(const uint32_t *edges, uint64_t n, uint64_t m, uint32_t r,
                    uint32_t *order, uint32_t *claim, uint64_t *layer_off,
                    uint64_t max_layers, uint32_t *rounds, uint64_t *n_peeled)
{
    return peel_rounds_impl(edges, n, m, r, order, claim, layer_off, max_layers, rounds,
                            n_peeled, 0);
}

/* The same round-synchronous peel for a general (not r-partite) hypergraph
 * on [0, m): the hinge is the smallest position j of the edge's row whose
 * vertex has degree 1 in the edge's round. */
int orc_peel_rounds_general(const uint32_t *edges, uint64_t n, uint64_t m, uint32_t r,
                            uint32_t *order, uint32_t *claim, uint64_t *layer_off,
                            uint64_t max_layers, uint32_t *rounds, uint64_t *n_peeled)
{
    return peel_rounds_impl(edges, n, m, r, order, claim, layer_off, max_layers, rounds,
                            n_peeled, 1);
}

/* Edges of a general r-hypergraph: vertex j of key k is mix64(k ^ (seed +
 * j)) mod m, any vertex in any position (sec. 3's h_j: S -> [gamma n]). */
int orc_hash_edges_general(const uint64_t *keys, uint64_t n, uint64_t m, uint32_t r,
                           uint64_t seed, uint32_t *edges)
{
    if (r < 2 || r > ORC_MAX_R || m == 0 || m >= (1ull << 32))
        return ORC_EINVAL;
    for (uint64_t i = 0; i < n; i++)
        for (uint32_t j = 0; j < r; j++)
            edges[i * r + j] = (uint32_t)(orc_mix64(keys[i] ^ (seed + j)) % m);
    return ORC_OK;
}

/* Standard linear-time greedy peel (sec. 1, sec. 3), with the packed
 * incidence list in place of explicit lists ("Standard+XOR", sec. 5): take
 * a vertex of degree 1, remove its only edge, repeat.  A LIFO stack holds
 * the candidate vertices.  order[0 .. *n_peeled) is the removal order (a
 * peeling order, not the canonical one); peeled[e] = 1 for removed edges.
 * The set of removed edges is the complement of the unique 2-core. */
int orc_peel_greedy(const uint32_t *edges, uint64_t n, uint64_t m, uint32_t r,
                    uint32_t *order, uint8_t *peeled, uint64_t *n_peeled)
{
    if (r < 2 || r > ORC_MAX_R || n >= (1ull << 32))
        return ORC_EINVAL;
    *n_peeled = 0;
    if (n == 0)
        return ORC_OK;
    int rc = ORC_OK;
    uint32_t *deg = malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t *x = malloc((m ? m : 1) * sizeof(uint32_t));
    /* each vertex is pushed at most once initially plus once per decrement */
    uint64_t cap = m + n * r + 1;
    uint32_t *stack = malloc(cap * sizeof(uint32_t));
    if (!deg || !x || !stack) {
        rc = ORC_ENOMEM;
        goto out;
    }
    rc = orc_incidence(edges, n, m, r, deg, x);
    if (rc)
        goto out;
    memset(peeled, 0, n);
    uint64_t sp = 0;
    for (uint64_t v = 0; v < m; v++)
        if (deg[v] == 1)
            stack[sp++] = (uint32_t)v;
    uint64_t cnt = 0;
    while (sp > 0) {
        uint32_t v = stack[--sp];
        if (deg[v] != 1)
            continue;
        uint32_t e = x[v];
        if (peeled[e]) {
            rc = ORC_EINTERNAL;
            goto out;
        }
        peeled[e] = 1;
        order[cnt++] = e;
        for (uint32_t j = 0; j < r; j++) {
            uint32_t w = edges[(uint64_t)e * r + j];
            deg[w] -= 1;
            x[w] ^= e;
            if (deg[w] == 1)
                stack[sp++] = w;
        }
    }
    *n_peeled = cnt;
out:
    free(deg);
    free(x);
    free(stack);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Validator: explicit incidence lists (not the XOR trick).              */
/* ---------------------------------------------------------------------- */

/* Checks, with explicit per-vertex incidence lists (CSR):
 *  1. order is a permutation of [0, n);
 *  2. each of the first n_peeled edges has a vertex of degree 1 in the
 *     graph left after removing the edges before it (sec. 1 definition of
 *     a peeling order);
 *  3. the remaining n - n_peeled edges have no vertex of degree 1 among
 *     them, i.e. they form a 2-core (sec. 1), so the peel is maximal.
 * If claim != NULL, also checks the layered structure of sec. 4.2:
 *  4. the rounds claim >> 2 along order are 0, ..., 0, 1, ..., R-1 with no
 *     gap, and at the start of round t every vertex of degree 1 has its one
 *     alive edge in layer t (the layer is every edge a degree-1 vertex
 *     retrieves, not a subset);
 *  5. hinge = claim & 3 is the smallest position whose vertex has degree 1
 *     at the start of the edge's round (so every edge of the layer has a
 *     degree-1 vertex); core edges carry ORC_UNCLAIMED.
 * The degree-1 vertices at the start of round t + 1 are found among the
 * vertices touched by round t (a vertex of degree 1 at the start of round
 * t that keeps it would already fail check 4).
 * Returns 0 when every check passes, otherwise a positive code naming the
 * first failed check (10 * check + detail). */
int orc_validate(const uint32_t *edges, uint64_t n, uint64_t m, uint32_t r,
                 const uint32_t *order, uint64_t n_peeled,
                 const uint32_t *claim)
{
    if (r < 2 || r > ORC_MAX_R || n_peeled > n)
        return ORC_EINVAL;
    int rc = 0;
    uint64_t *start = calloc(m + 1, sizeof(uint64_t));
    uint32_t *adj = malloc((n * r + 1) * sizeof(uint32_t));
    uint32_t *deg = calloc(m + 1, sizeof(uint32_t));
    uint8_t *alive = malloc(n + 1);
    uint8_t *seen = calloc(n + 1, 1);
    uint64_t *fill = calloc(m + 1, sizeof(uint64_t));
    uint32_t *cand = malloc((m + n * r + 1) * sizeof(uint32_t));
    if (!start || !adj || !deg || !alive || !seen || !fill || !cand) {
        rc = ORC_ENOMEM;
        goto out;
    }
    for (uint64_t e = 0; e < n; e++)
        for (uint32_t j = 0; j < r; j++) {
            uint32_t v = edges[e * r + j];
            if (v >= m) {
                rc = 11;
                goto out;
            }
            start[v + 1] += 1;
        }
    for (uint64_t v = 0; v < m; v++)
        start[v + 1] += start[v];
    for (uint64_t e = 0; e < n; e++)
        for (uint32_t j = 0; j < r; j++) {
            uint32_t v = edges[e * r + j];
            adj[start[v] + fill[v]++] = (uint32_t)e;
            deg[v] += 1;
        }
    /* 1. permutation */
    for (uint64_t k = 0; k < n; k++) {
        if (order[k] >= n || seen[order[k]]) {
            rc = 12;
            goto out;
        }
        seen[order[k]] = 1;
    }
    memset(alive, 1, n);
    if (!claim) {
        /* 2. peeling-order property, one edge at a time */
        for (uint64_t q = 0; q < n_peeled; q++) {
            uint32_t e = order[q];
            int ok = 0;
            for (uint32_t j = 0; j < r; j++)
                if (deg[edges[(uint64_t)e * r + j]] == 1)
                    ok = 1;
            if (!ok) {
                rc = 21;
                goto out;
            }
            alive[e] = 0;
            for (uint32_t j = 0; j < r; j++)
                deg[edges[(uint64_t)e * r + j]] -= 1;
        }
    } else {
        uint64_t nc = 0;
        for (uint64_t v = 0; v < m; v++)
            if (deg[v] == 1)
                cand[nc++] = (uint32_t)v;
        uint64_t k = 0;
        uint32_t t = 0;
        while (k < n_peeled) {
            uint32_t c0 = claim[order[k]];
            if (c0 == ORC_UNCLAIMED || (c0 >> 2) != t) {
                rc = 41;
                goto out;
            }
            uint64_t k_end = k;
            while (k_end < n_peeled && claim[order[k_end]] != ORC_UNCLAIMED &&
                   (claim[order[k_end]] >> 2) == t)
                k_end++;
            /* 4. every degree-1 vertex retrieves an edge of this layer */
            for (uint64_t c = 0; c < nc; c++) {
                uint32_t v = cand[c];
                if (deg[v] != 1)
                    continue;
                uint32_t ee = ORC_UNCLAIMED;
                for (uint64_t a = start[v]; a < start[v + 1]; a++)
                    if (alive[adj[a]])
                        ee = adj[a];
                if (ee == ORC_UNCLAIMED) {
                    rc = 43;
                    goto out;
                }
                if (claim[ee] == ORC_UNCLAIMED || (claim[ee] >> 2) != t) {
                    rc = 44;
                    goto out;
                }
            }
            /* 5. hinges of the layer, against degrees at round start */
            for (uint64_t q = k; q < k_end; q++) {
                uint32_t e = order[q];
                uint32_t h = ORC_UNCLAIMED;
                for (uint32_t j = 0; j < r; j++)
                    if (deg[edges[(uint64_t)e * r + j]] == 1) {
                        h = j;
                        break;
                    }
                if (h != (claim[e] & 3u)) {
                    rc = 51;
                    goto out;
                }
            }
            /* remove the layer; its vertices are the next candidates */
            nc = 0;
            for (uint64_t q = k; q < k_end; q++) {
                uint32_t e = order[q];
                alive[e] = 0;
                for (uint32_t j = 0; j < r; j++) {
                    uint32_t w = edges[(uint64_t)e * r + j];
                    deg[w] -= 1;
                    cand[nc++] = w;
                }
            }
            k = k_end;
            t += 1;
        }
        /* no further round: no vertex has degree 1 after the last layer */
        for (uint64_t c = 0; c < nc; c++)
            if (deg[cand[c]] == 1) {
                rc = 45;
                goto out;
            }
    }
    /* 3. what is left is a 2-core */
    for (uint64_t q = n_peeled; q < n; q++) {
        uint32_t e = order[q];
        if (claim && claim[e] != ORC_UNCLAIMED) {
            rc = 52;
            goto out;
        }
        for (uint32_t j = 0; j < r; j++)
            if (deg[edges[(uint64_t)e * r + j]] < 2) {
                rc = 31;
                goto out;
            }
    }
out:
    free(start);
    free(adj);
    free(deg);
    free(alive);
    free(seen);
    free(fill);
    free(cand);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* MWHC assignment, rank and lookup (sec. 3, sec. 4.3 "Avoiding backward  */
/* scans", sec. 5 broadword rank).                                        */
/* ---------------------------------------------------------------------- */

static uint32_t g_get(const uint64_t *G, uint64_t v)
{
    return (uint32_t)((G[v >> 5] >> (2 * (v & 31))) & 3u);
}

static void g_set(uint64_t *G, uint64_t v, uint32_t val)
{
    G[v >> 5] |= (uint64_t)(val & 3u) << (2 * (v & 31));
}

/* Solve u_{h0} + u_{h1} + u_{h2} = f(x) (mod 3) with f(x) = hinge, for
 * r = 3, visiting layers from the last to the first and each layer in its
 * stored order: for an edge e with hinge h, the hinge vertex is the only
 * one of e not fixed yet, so u at the hinge = (h - sum of the other two)
 * mod 3.  A value 0 is stored as 3.  G has ceil(m / 32) words. */
int orc_mphf_assign(const uint32_t *edges, uint64_t n, uint64_t m,
                    const uint32_t *order, const uint32_t *claim,
                    const uint64_t *layer_off, uint32_t rounds, uint64_t *G)
{
    (void)n;
    uint64_t words = (m + 31) / 32;
    memset(G, 0, words * sizeof(uint64_t));
    for (int64_t t = (int64_t)rounds - 1; t >= 0; t--) {
        for (uint64_t q = layer_off[t]; q < layer_off[t + 1]; q++) {
            uint32_t e = order[q];
            uint32_t h = claim[e] & 3u;
            if (claim[e] == ORC_UNCLAIMED || h >= 3)
                return ORC_EINTERNAL;
            uint32_t s = 0;
            for (uint32_t j = 0; j < 3; j++)
                if (j != h)
                    s += g_get(G, edges[(uint64_t)e * 3 + j]);
            uint32_t val = (h + 3 * 3 - (s % 3)) % 3;
            if (g_get(G, edges[(uint64_t)e * 3 + h]) != 0)
                return ORC_EINTERNAL; /* a hinge is assigned once */
            g_set(G, edges[(uint64_t)e * 3 + h], val ? val : 3u);
        }
    }
    return ORC_OK;
}

/* Rank directory: dir[b] = number of non-zero 2-bit values among vertices
 * [0, 512 b), for b = 0 .. ceil(m / 512).  Counted one vertex at a time. */
int orc_rank_dir(const uint64_t *G, uint64_t m, uint64_t *dir)
{
    uint64_t blocks = (m + 511) / 512;
    uint64_t c = 0;
    for (uint64_t b = 0; b < blocks; b++) {
        dir[b] = c;
        for (uint64_t v = b * 512; v < (b + 1) * 512 && v < m; v++)
            if (g_get(G, v) != 0)
                c += 1;
    }
    dir[blocks] = c;
    return ORC_OK;
}

/* Lookup of a key (sec. 3 and sec. 5): i = (G[v0] + G[v1] + G[v2]) mod 3,
 * result = rank of v_i = number of assigned vertices before v_i. */
uint64_t orc_lookup(uint64_t key, uint64_t seed, uint64_t m, const uint64_t *G,
                    const uint64_t *dir)
{
    uint64_t P = m / 3;
    uint32_t v[3];
    uint32_t s = 0;
    for (uint32_t j = 0; j < 3; j++) {
        v[j] = (uint32_t)(orc_mix64(key ^ (seed + j)) % P + (uint64_t)j * P);
        s += g_get(G, v[j]);
    }
    uint32_t i = s % 3;
    uint64_t b = v[i] / 512;
    uint64_t rank = dir[b];
    for (uint64_t u = b * 512; u < v[i]; u++)
        if (g_get(G, u) != 0)
            rank += 1;
    return rank;
}

/* Whole MPHF build (sec. 3): hash with seed, seed + 1, ... until the graph
 * peels completely (at most max_tries hash seeds), then assign and rank.
 * Outputs G[ceil(m / 32)], dir[ceil(m / 512) + 1], *seed_used, *rounds. */
int orc_mphf_build(const uint64_t *keys, uint64_t n, uint64_t seed,
                   uint32_t gamma_milli, uint32_t max_tries, uint64_t *G,
                   uint64_t *dir, uint64_t *seed_used, uint32_t *rounds_out)
{
    uint64_t m = orc_num_vertices(n, gamma_milli, 3);
    if (m >= (1ull << 32) || n >= (1ull << 32))
        return ORC_EINVAL;
    int rc = ORC_ERETRIES;
    uint32_t *edges = malloc((n * 3 + 1) * sizeof(uint32_t));
    uint32_t *order = malloc((n + 1) * sizeof(uint32_t));
    uint32_t *claim = malloc((n + 1) * sizeof(uint32_t));
    uint64_t max_layers = n + 1;
    uint64_t *loff = malloc((max_layers + 1) * sizeof(uint64_t));
    if (!edges || !order || !claim || !loff) {
        rc = ORC_ENOMEM;
        goto out;
    }
    for (uint32_t a = 0; a < max_tries; a++) {
        uint64_t s = seed + a;
        int e1 = orc_hash_edges(keys, n, m, 3, s, edges);
        if (e1) {
            rc = e1;
            goto out;
        }
        uint32_t rounds = 0;
        uint64_t peeled = 0;
        int e2 = orc_peel_rounds(edges, n, m, 3, order, claim, loff, max_layers,
                                 &rounds, &peeled);
        if (e2) {
            rc = e2;
            goto out;
        }
        if (peeled < n)
            continue;
        orc_mphf_assign(edges, n, m, order, claim, loff, rounds, G);
        orc_rank_dir(G, m, dir);
        *seed_used = s;
        if (rounds_out)
            *rounds_out = rounds;
        rc = ORC_OK;
        break;
    }
out:
    free(edges);
    free(order);
    free(claim);
    free(loff);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Static functions (sec. 3): any f: S -> [sigma] is stored as an array u  */
/* of gamma n values in [sigma] with f(x) = u[h0(x)] + u[h1(x)] + u[h2(x)] */
/* mod sigma, ceil(log2 sigma) bits per value.  The MPHF above is the case */
/* sigma = 3 with f(x) = hinge position (plus its "0 stored as 3" code).   */
/* ---------------------------------------------------------------------- */

/* ceil(log2 sigma): bits per stored value (sigma >= 2). */
uint32_t orc_sf_bits(uint64_t sigma)
{
    uint32_t b = 0;
    while (b < 64 && (1ull << b) < sigma)
        b++;
    return b;
}

/* u[v] occupies bits [v b, (v + 1) b) of the bit string U, bit i of the
 * string being bit (i mod 64) of word i / 64; read and written one bit at a
 * time. */
static uint64_t u_get(const uint64_t *U, uint64_t v, uint32_t b)
{
    uint64_t x = 0;
    for (uint32_t i = 0; i < b; i++) {
        uint64_t bit = v * b + i;
        x |= ((U[bit >> 6] >> (bit & 63)) & 1u) << i;
    }
    return x;
}

static void u_put(uint64_t *U, uint64_t v, uint32_t b, uint64_t x)
{
    for (uint32_t i = 0; i < b; i++) {
        uint64_t bit = v * b + i;
        uint64_t mask = 1ull << (bit & 63);
        if ((x >> i) & 1u)
            U[bit >> 6] |= mask;
        else
            U[bit >> 6] &= ~mask;
    }
}

/* Words of the bit string for m values of b bits. */
uint64_t orc_sf_words(uint64_t m, uint32_t b)
{
    return (m * b + 63) / 64;
}

/* Solve u[h0] + u[h1] + u[h2] = values[e] (mod sigma) for every peeled edge
 * e (r = 3), layers from the last to the first: the hinge vertex of e is
 * the only one of e not fixed yet, so it takes (values[e] - the other two)
 * mod sigma; vertices never a hinge keep 0.  values[e] >= sigma is an
 * error (ORC_EINVAL). */
int orc_sf_assign(const uint32_t *edges, uint64_t n, uint64_t m, const uint32_t *order,
                  const uint32_t *claim, const uint64_t *layer_off, uint32_t rounds,
                  const uint32_t *values, uint64_t sigma, uint64_t *U)
{
    (void)n;
    if (sigma < 2 || sigma > (1ull << 32))
        return ORC_EINVAL;
    uint32_t b = orc_sf_bits(sigma);
    memset(U, 0, orc_sf_words(m, b) * sizeof(uint64_t));
    for (int64_t t = (int64_t)rounds - 1; t >= 0; t--) {
        for (uint64_t q = layer_off[t]; q < layer_off[t + 1]; q++) {
            uint32_t e = order[q];
            if (claim[e] == ORC_UNCLAIMED)
                return ORC_EINTERNAL;
            uint32_t h = claim[e] & 3u;
            if (values[e] >= sigma)
                return ORC_EINVAL;
            uint64_t other = 0;
            for (uint32_t j = 0; j < 3; j++)
                if (j != h)
                    other += u_get(U, edges[(uint64_t)e * 3 + j], b);
            uint64_t val = ((uint64_t)values[e] + sigma - other % sigma) % sigma;
            u_put(U, edges[(uint64_t)e * 3 + h], b, val);
        }
    }
    return ORC_OK;
}

/* f(key) = (u[h0] + u[h1] + u[h2]) mod sigma. */
uint64_t orc_sf_lookup(uint64_t key, uint64_t seed, uint64_t m, uint64_t sigma,
                       const uint64_t *U)
{
    uint64_t P = m / 3;
    uint32_t b = orc_sf_bits(sigma);
    uint64_t s = 0;
    for (uint32_t j = 0; j < 3; j++) {
        uint64_t v = orc_mix64(key ^ (seed + j)) % P + (uint64_t)j * P;
        s += u_get(U, v, b);
    }
    return s % sigma;
}

/* Whole static-function build (sec. 3): hash with seed, seed + 1, ... until
 * the graph peels completely (at most max_tries seeds), then assign.
 * U has orc_sf_words(m, ceil(log2 sigma)) words. */
int orc_sf_build(const uint64_t *keys, const uint32_t *values, uint64_t n, uint64_t sigma,
                 uint64_t seed, uint32_t gamma_milli, uint32_t max_tries, uint64_t *U,
                 uint64_t *seed_used, uint32_t *rounds_out)
{
    uint64_t m = orc_num_vertices(n, gamma_milli, 3);
    if (m >= (1ull << 32) || n >= (1ull << 32) || sigma < 2 || sigma > (1ull << 32))
        return ORC_EINVAL;
    int rc = ORC_ERETRIES;
    uint32_t *edges = malloc((n * 3 + 1) * sizeof(uint32_t));
    uint32_t *order = malloc((n + 1) * sizeof(uint32_t));
    uint32_t *claim = malloc((n + 1) * sizeof(uint32_t));
    uint64_t max_layers = n + 1;
    uint64_t *loff = malloc((max_layers + 1) * sizeof(uint64_t));
    if (!edges || !order || !claim || !loff) {
        rc = ORC_ENOMEM;
        goto out;
    }
    for (uint32_t a = 0; a < max_tries; a++) {
        uint64_t s = seed + a;
        int e1 = orc_hash_edges(keys, n, m, 3, s, edges);
        if (e1) {
            rc = e1;
            goto out;
        }
        uint32_t rounds = 0;
        uint64_t peeled = 0;
        int e2 = orc_peel_rounds(edges, n, m, 3, order, claim, loff, max_layers,
                                 &rounds, &peeled);
        if (e2) {
            rc = e2;
            goto out;
        }
        if (peeled < n)
            continue;
        rc = orc_sf_assign(edges, n, m, order, claim, loff, rounds, values, sigma, U);
        if (rc == ORC_OK) {
            *seed_used = s;
            if (rounds_out)
                *rounds_out = rounds;
        }
        break;
    }
out:
    free(edges);
    free(order);
    free(claim);
    free(loff);
    return rc;
}
