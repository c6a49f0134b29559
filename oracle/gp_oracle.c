/*
 * gp_oracle.c -- plain, single-threaded CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Every step is the obvious sequential loop.  Where the method is parallel
 * (matching picks, gain computation, moves), the oracle reads the state at the
 * start of the step and writes the new state afterwards, so its results are
 * those of the synchronous step regardless of loop order.
 *
 * Paper passages this follows (Wu, Lohmann, Schroeder-Preikschat):
 *   Sec. III.B  weighted DAG (kernel times on vertices, transfer time on
 *               edges, the same time in either direction), workload ratio
 *               Eq. (1)-(2), two partitions;
 *   Sec. IV.C   the policy keeps the load balanced and minimises the cut
 *               transfer cost;
 *   Sec. IV.C   (matrix-multiply discussion) a large speed gap leaves ~0 work
 *               on the CPU.
 * Everything below the partition objective (the multilevel algorithm) is not
 * in the paper, which delegates it to METIS; the comments state the reading.
 */
#include "gp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* ------------------------------------------------------------------------ */
/* splitmix64 finaliser (Vigna, public domain) and the edge hash.            */
/* ------------------------------------------------------------------------ */
uint64_t og_mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ULL;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebULL;
  z ^= z >> 31;
  return z;
}

/* h(seed, a, b) = mix64(seed XOR mix64(a << 32 | b)) */
uint64_t og_hash(uint64_t seed, uint32_t a, uint32_t b) {
  return og_mix64(seed ^ og_mix64(((uint64_t)a << 32) | (uint64_t)b));
}

/* ------------------------------------------------------------------------ */
/* Input validation.  Precedence of the error codes: INVALID, then OVERFLOW, */
/* then NOT_DAG (a self-loop is a cycle of length one).                      */
/* ------------------------------------------------------------------------ */
#define OG_MAX_N (((int64_t)1 << 31) - 2)

static int og_is_acyclic(int64_t n, const int64_t* off, const int32_t* cols) {
  int64_t* indeg = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!indeg || !queue) {
    free(indeg);
    free(queue);
    return -1;
  }
  for (int64_t e = 0; e < off[n]; e++) indeg[cols[e]]++;
  int64_t head = 0, tail = 0;
  for (int64_t v = 0; v < n; v++)
    if (indeg[v] == 0) queue[tail++] = (int32_t)v;
  while (head < tail) {
    int32_t v = queue[head++];
    for (int64_t e = off[v]; e < off[v + 1]; e++)
      if (--indeg[cols[e]] == 0) queue[tail++] = cols[e];
  }
  free(indeg);
  free(queue);
  return tail == n ? 1 : 0;
}

int og_validate(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                const int32_t* cC, const int32_t* cG) {
  if (n < 0 || m < 0 || n > OG_MAX_N) return OG_ERR_INVALID;
  if (off[0] != 0 || off[n] != m) return OG_ERR_INVALID;
  for (int64_t v = 0; v < n; v++)
    if (off[v + 1] < off[v]) return OG_ERR_INVALID;
  for (int64_t e = 0; e < m; e++)
    if (cols[e] < 0 || cols[e] >= n || w[e] < 0) return OG_ERR_INVALID;
  for (int64_t v = 0; v < n; v++)
    if (cC[v] < 0 || cG[v] < 0) return OG_ERR_INVALID;
  i128 sw = 0, sc = 0, sg = 0;
  for (int64_t e = 0; e < m; e++) sw += w[e];
  for (int64_t v = 0; v < n; v++) {
    sc += cC[v];
    sg += cG[v];
  }
  if (sw > OG_SUM_LIMIT || sc > OG_SUM_LIMIT || sg > OG_SUM_LIMIT) return OG_ERR_OVERFLOW;
  for (int64_t v = 0; v < n; v++)
    for (int64_t e = off[v]; e < off[v + 1]; e++)
      if (cols[e] == v) return OG_ERR_NOT_DAG;
  int acyc = og_is_acyclic(n, off, cols);
  if (acyc < 0) return OG_ERR_OOM;
  return acyc ? OG_OK : OG_ERR_NOT_DAG;
}

/* ------------------------------------------------------------------------ */
/* Balance bounds from Eq. (1)-(2), in exact integers.                       */
/*                                                                           */
/* Eq. (1) gives the CPU its share R_CPU = T_GPU / (T_GPU + T_CPU) of the     */
/* work and Eq. (2) the GPU the rest.  With the summed kernel times SC (all   */
/* on the CPU) and SG (all on the GPU), the CPU's load at that share is       */
/* SC * SG / (SC + SG) = T*, and the GPU's load is the same T*.  Each side     */
/* may exceed T* by the tolerance:  B = floor(T* (1e6 + tol_ppm) / 1e6).      */
/* An explicit ratio r replaces Eq. (1): B_C from SC * r, B_G from SG (1 - r), */
/* with r quantised to 32 fraction bits.                                      */
/* ------------------------------------------------------------------------ */
int og_bounds(int64_t SC, int64_t SG, double r_cpu, double tol, int64_t* BC, int64_t* BG) {
  if (!(tol >= 0.0 && tol <= 1.0)) return OG_ERR_INVALID;
  if (isnan(r_cpu) || r_cpu > 1.0) return OG_ERR_INVALID;
  if (SC < 0 || SG < 0) return OG_ERR_INVALID;
  const i128 ppm = (i128)llround(tol * 1e6);
  const i128 scale = (i128)1000000 + ppm;
  if (r_cpu < 0.0) {
    const i128 den = (i128)SC + (i128)SG;
    const i128 tstar = den == 0 ? 0 : ((i128)SC * (i128)SG) / den;
    *BC = (int64_t)((tstar * scale) / 1000000);
    *BG = *BC;
  } else {
    const i128 rq = (i128)llround(r_cpu * 4294967296.0);
    const i128 tc = ((i128)SC * rq) >> 32;
    const i128 tg = ((i128)SG * (((i128)1 << 32) - rq)) >> 32;
    *BC = (int64_t)((tc * scale) / 1000000);
    *BG = (int64_t)((tg * scale) / 1000000);
  }
  return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* Symmetrisation.  The cut is measured on the undirected graph because a     */
/* transfer costs the same in both directions (Sec. III.B): every directed    */
/* entry u->v of weight w adds w to W(u,v) and to W(v,u).  Parallel entries   */
/* add up.  Rows are sorted by neighbour id.                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t w;
  int32_t col;
} og_entry;

static int og_cmp_entry(const void* a, const void* b) {
  const og_entry* x = (const og_entry*)a;
  const og_entry* y = (const og_entry*)b;
  return (x->col > y->col) - (x->col < y->col);
}

/* Sort a row's entries by neighbour and add up equal neighbours; returns the
 * number of distinct entries left at the front of the array. */
static int64_t og_sort_merge(og_entry* e, int64_t len) {
  if (len == 0) return 0;
  qsort(e, (size_t)len, sizeof(og_entry), og_cmp_entry);
  int64_t k = 0;
  for (int64_t i = 1; i < len; i++) {
    if (e[i].col == e[k].col)
      e[k].w += e[i].w;
    else
      e[++k] = e[i];
  }
  return k + 1;
}

int og_symmetrize(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                  int64_t* uoff, int32_t* uadj, int64_t* uW, int64_t* a_out) {
  int64_t* rawoff = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  og_entry* raw = (og_entry*)malloc((size_t)(2 * m + 1) * sizeof(og_entry));
  if (!rawoff || !fill || !raw) {
    free(rawoff);
    free(fill);
    free(raw);
    return OG_ERR_OOM;
  }
  for (int64_t v = 0; v < n; v++) rawoff[v + 1] += off[v + 1] - off[v];
  for (int64_t e = 0; e < m; e++) rawoff[(int64_t)cols[e] + 1] += 1;
  for (int64_t v = 0; v < n; v++) rawoff[v + 1] += rawoff[v];
  for (int64_t v = 0; v < n; v++) fill[v] = rawoff[v];
  for (int64_t u = 0; u < n; u++) {
    for (int64_t e = off[u]; e < off[u + 1]; e++) {
      int32_t v = cols[e];
      raw[fill[u]].col = v;
      raw[fill[u]].w = w[e];
      fill[u]++;
      raw[fill[v]].col = (int32_t)u;
      raw[fill[v]].w = w[e];
      fill[v]++;
    }
  }
  int64_t a = 0;
  uoff[0] = 0;
  for (int64_t v = 0; v < n; v++) {
    int64_t len = og_sort_merge(raw + rawoff[v], rawoff[v + 1] - rawoff[v]);
    for (int64_t i = 0; i < len; i++) {
      uadj[a] = raw[rawoff[v] + i].col;
      uW[a] = raw[rawoff[v] + i].w;
      a++;
    }
    uoff[v + 1] = a;
  }
  *a_out = a;
  free(rawoff);
  free(fill);
  free(raw);
  return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* Coarsening step 1: handshake heavy-edge matching.                          */
/*                                                                           */
/* `rounds` synchronous rounds.  In a round every unmatched vertex v looks at  */
/* its unmatched neighbours u whose merged weights stay within the caps        */
/* (vC[v]+vC[u] <= cap_cpu and vG[v]+vG[u] <= cap_gpu) and picks the one whose */
/* edge is largest under the key (W desc, h(seed,min,max) desc, min asc,       */
/* max asc), min/max being the smaller/larger endpoint id.  v and u are        */
/* matched when each picked the other.  Picks are all made from the matching  */
/* state at the start of the round.  mate[v] = partner or -1.                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t W;
  uint64_t h;
  uint32_t mn, mx;
  int32_t u;
} og_edge_key;

/* 1 if x ranks above y */
static int og_key_better(const og_edge_key* x, const og_edge_key* y) {
  if (x->W != y->W) return x->W > y->W;
  if (x->h != y->h) return x->h > y->h;
  if (x->mn != y->mn) return x->mn < y->mn;
  return x->mx < y->mx;
}

/* Fixed vertices (the paper's host-source kernel, Sec. III.B, generalised): fix[v] = 0 pins v to the
 * CPU, 1 to the GPU, -1 leaves it free; fix == NULL means every vertex is free.  Two vertices may merge
 * unless they are pinned to different sides; a coarse vertex is pinned where either member is. */
static int og_compatible(const int8_t* fix, int64_t a, int64_t b) {
  return !fix || fix[a] < 0 || fix[b] < 0 || fix[a] == fix[b];
}

static int og_match_fix(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                        const int64_t* vC, const int64_t* vG, const int8_t* fix, int64_t capC,
                        int64_t capG, uint64_t seed, int32_t rounds, int32_t* mate) {
  int32_t* pick = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!pick) return OG_ERR_OOM;
  for (int64_t v = 0; v < n; v++) mate[v] = -1;
  for (int32_t r = 0; r < rounds; r++) {
    for (int64_t v = 0; v < n; v++) {
      pick[v] = -1;
      if (mate[v] != -1) continue;
      og_edge_key best;
      int have = 0;
      for (int64_t e = off[v]; e < off[v + 1]; e++) {
        const int32_t u = adj[e];
        if (mate[u] != -1) continue;
        if (vC[v] + vC[u] > capC || vG[v] + vG[u] > capG) continue;
        if (!og_compatible(fix, v, u)) continue;
        og_edge_key k;
        k.W = W[e];
        k.mn = (uint32_t)(v < u ? v : u);
        k.mx = (uint32_t)(v < u ? u : v);
        k.h = og_hash(seed, k.mn, k.mx);
        k.u = u;
        if (!have || og_key_better(&k, &best)) {
          best = k;
          have = 1;
        }
      }
      if (have) pick[v] = best.u;
    }
    /* confirm: reads only the picks of this round */
    for (int64_t v = 0; v < n; v++) {
      const int32_t u = pick[v];
      if (u >= 0 && pick[u] == (int32_t)v) mate[v] = u;
    }
  }
  free(pick);
  return OG_OK;
}

int og_match(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
             const int64_t* vC, const int64_t* vG, int64_t capC, int64_t capG, uint64_t seed,
             int32_t rounds, int32_t* mate) {
  return og_match_fix(n, off, adj, W, vC, vG, NULL, capC, capG, seed, rounds, mate);
}

/* ------------------------------------------------------------------------ */
/* Coarsening step 1b: two-hop pairing of the vertices the handshake rounds   */
/* left unmatched.                                                           */
/*                                                                           */
/* After a few handshake rounds, coarse graphs fill up with light vertices    */
/* whose neighbours are all matched heavy vertices ("satellites" of a hub);   */
/* no handshake round can ever pair them and coarsening stalls.  Each         */
/* unmatched vertex therefore names an anchor: its best neighbour under the   */
/* matching key, over all neighbours.  Walking each vertex h's row in         */
/* ascending neighbour order, the unmatched vertices anchored at h are paired */
/* in turn: a vertex is paired with the pending one when their merged weights */
/* fit the caps, and otherwise becomes the pending one.  Paired vertices need */
/* not be adjacent.  Anchors are all chosen before any pairing.              */
/* ------------------------------------------------------------------------ */
static int og_match_twohop_fix(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                               const int64_t* vC, const int64_t* vG, const int8_t* fix, int64_t capC,
                               int64_t capG, uint64_t seed, int32_t* mate) {
  int32_t* anchor = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!anchor) return OG_ERR_OOM;
  for (int64_t v = 0; v < n; v++) {
    anchor[v] = -1;
    if (mate[v] != -1) continue;
    og_edge_key best;
    int have = 0;
    for (int64_t e = off[v]; e < off[v + 1]; e++) {
      const int32_t u = adj[e];
      og_edge_key k;
      k.W = W[e];
      k.mn = (uint32_t)(v < u ? v : u);
      k.mx = (uint32_t)(v < u ? u : v);
      k.h = og_hash(seed, k.mn, k.mx);
      k.u = u;
      if (!have || og_key_better(&k, &best)) {
        best = k;
        have = 1;
      }
    }
    if (have) anchor[v] = best.u;
  }
  for (int64_t h = 0; h < n; h++) {
    int32_t pending = -1;
    for (int64_t e = off[h]; e < off[h + 1]; e++) {
      const int32_t v = adj[e];
      if (anchor[v] != (int32_t)h) continue;
      if (pending >= 0 && vC[pending] + vC[v] <= capC && vG[pending] + vG[v] <= capG &&
          og_compatible(fix, pending, v)) {
        mate[pending] = v;
        mate[v] = pending;
        pending = -1;
      } else {
        pending = v;
      }
    }
  }
  free(anchor);
  return OG_OK;
}

int og_match_twohop(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                    const int64_t* vC, const int64_t* vG, int64_t capC, int64_t capG,
                    uint64_t seed, int32_t* mate) {
  return og_match_twohop_fix(n, off, adj, W, vC, vG, NULL, capC, capG, seed, mate);
}

/* Number of coarse vertices the matching yields: one per unmatched vertex and
 * one per matched pair. */
int64_t og_count_coarse(int64_t n, const int32_t* mate) {
  int64_t c = 0;
  for (int64_t v = 0; v < n; v++)
    if (mate[v] < 0 || v < mate[v]) c++;
  return c;
}

/* ------------------------------------------------------------------------ */
/* Coarsening step 2: contraction.                                            */
/*                                                                           */
/* The representative of a coarse vertex is its smaller member.  Coarse ids   */
/* number the representatives in vertex order; the partner takes the same id. */
/* Coarse vertex weights are the sums of the members' weights.  A coarse row   */
/* is the union of both members' rows mapped through cmap, without the coarse */
/* vertex itself, equal neighbours added up, sorted by id.                    */
/* ------------------------------------------------------------------------ */
int og_contract(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                const int64_t* vC, const int64_t* vG, const int32_t* mate, int32_t* cmap,
                int64_t* nc_out, int64_t* coff, int32_t* cadj, int64_t* cW, int64_t* cvC,
                int64_t* cvG, int64_t* ac_out) {
  int64_t nc = 0;
  for (int64_t v = 0; v < n; v++)
    if (mate[v] < 0 || v < mate[v]) cmap[v] = (int32_t)nc++;
  for (int64_t v = 0; v < n; v++)
    if (!(mate[v] < 0 || v < mate[v])) cmap[v] = cmap[mate[v]];
  int64_t maxlen = 0;
  for (int64_t v = 0; v < n; v++) {
    int64_t len = off[v + 1] - off[v];
    if (mate[v] >= 0) len += off[mate[v] + 1] - off[mate[v]];
    if (len > maxlen) maxlen = len;
  }
  og_entry* buf = (og_entry*)malloc((size_t)(maxlen + 1) * sizeof(og_entry));
  if (!buf) return OG_ERR_OOM;
  int64_t a = 0;
  coff[0] = 0;
  for (int64_t v = 0; v < n; v++) {
    if (!(mate[v] < 0 || v < mate[v])) continue;
    const int32_t c = cmap[v];
    int64_t len = 0;
    int64_t members[2] = {v, mate[v]};
    cvC[c] = 0;
    cvG[c] = 0;
    for (int k = 0; k < 2; k++) {
      const int64_t x = members[k];
      if (x < 0) continue;
      cvC[c] += vC[x];
      cvG[c] += vG[x];
      for (int64_t e = off[x]; e < off[x + 1]; e++) {
        const int32_t t = cmap[adj[e]];
        if (t == c) continue;
        buf[len].col = t;
        buf[len].w = W[e];
        len++;
      }
    }
    len = og_sort_merge(buf, len);
    for (int64_t i = 0; i < len; i++) {
      cadj[a] = buf[i].col;
      cW[a] = buf[i].w;
      a++;
    }
    coff[c + 1] = a;
  }
  free(buf);
  *nc_out = nc;
  *ac_out = a;
  return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* Initial bipartition: greedy graph growing (GGGP) on the coarsest graph.    */
/*                                                                           */
/* If everything fits on the GPU (sum vG <= B_G), the split is all-GPU: the   */
/* CPU gets no work, as the paper's matrix-multiply case shows for a large    */
/* speed gap (Sec. IV.C).  Otherwise 8 trials grow a CPU region from a hashed */
/* start vertex s_t = h(seed, 0xFFFFFFFF, t) mod n, all others on the GPU:     */
/*   - s_t moves to the CPU if its CPU weight fits under B_C;                 */
/*   - while the GPU is over B_G: among GPU-side vertices whose CPU weight    */
/*     still fits, take those adjacent to the CPU region (all of them when    */
/*     none is adjacent) and move the one with the largest gain              */
/*     W(to CPU) - W(to GPU), smallest id on ties; stop when none fits.       */
/* The best trial is the feasible one with the smallest cut, then the         */
/* smallest t.  trial_out = winning t, or -1 for the all-GPU split.           */
/* ------------------------------------------------------------------------ */
/* One trial: grow a CPU region from `start` (all others on the GPU).  side,
 * toC (W to the CPU region) and adjC (CPU neighbours) are caller scratch of
 * n entries; wsum[v] is v's total adjacency weight.  Returns the cut. */
/* With fixed vertices, the CPU-pinned ones start (and stay) in the CPU region, the GPU-pinned ones on
 * the GPU, and only free vertices move. */
static int64_t og_grow(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                       const int64_t* vC, const int64_t* vG, const int8_t* fix, const int64_t* wsum,
                       int64_t BC, int64_t BG, int64_t start, uint8_t* side, int64_t* toC,
                       int64_t* adjC, int64_t* LC_out, int64_t* LG_out) {
  int64_t LC = 0, LG = 0;
  for (int64_t v = 0; v < n; v++) {
    side[v] = (fix && fix[v] == 0) ? 0 : 1;
    toC[v] = 0;
    adjC[v] = 0;
  }
  for (int64_t v = 0; v < n; v++) {
    if (side[v] == 1) {
      LG += vG[v];
      continue;
    }
    LC += vC[v];
    for (int64_t e = off[v]; e < off[v + 1]; e++) {
      toC[adj[e]] += W[e];
      adjC[adj[e]] += 1;
    }
  }
  const int start_free = !fix || fix[start] < 0;
  int64_t x = (start_free && LC + vC[start] <= BC) ? start : -1;
  for (;;) {
    if (x >= 0) { /* move x to the CPU */
      side[x] = 0;
      LC += vC[x];
      LG -= vG[x];
      for (int64_t e = off[x]; e < off[x + 1]; e++) {
        toC[adj[e]] += W[e];
        adjC[adj[e]] += 1;
      }
    }
    if (LG <= BG) break;
    /* next vertex: adjacency class first, then gain, then smallest id */
    x = -1;
    int x_adj = 0;
    int64_t x_gain = 0;
    for (int64_t v = 0; v < n; v++) {
      if (side[v] != 1 || (fix && fix[v] >= 0) || LC + vC[v] > BC) continue;
      const int a = adjC[v] > 0;
      const int64_t g = 2 * toC[v] - wsum[v];
      if (x < 0 || a > x_adj || (a == x_adj && g > x_gain)) {
        x = v;
        x_adj = a;
        x_gain = g;
      }
    }
    if (x < 0) break;
  }
  int64_t cut = 0;
  for (int64_t v = 0; v < n; v++)
    if (side[v] == 0) cut += wsum[v] - toC[v];
  *LC_out = LC;
  *LG_out = LG;
  return cut;
}

int og_gggp_grow(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                 const int64_t* vC, const int64_t* vG, int64_t BC, int64_t BG, int64_t start,
                 uint8_t* part, int64_t* cut_out) {
  if (n <= 0 || start < 0 || start >= n) return OG_ERR_INVALID;
  int64_t* toC = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  int64_t* adjC = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  int64_t* wsum = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!toC || !adjC || !wsum) {
    free(toC);
    free(adjC);
    free(wsum);
    return OG_ERR_OOM;
  }
  for (int64_t v = 0; v < n; v++) {
    wsum[v] = 0;
    for (int64_t e = off[v]; e < off[v + 1]; e++) wsum[v] += W[e];
  }
  int64_t LC, LG;
  *cut_out = og_grow(n, off, adj, W, vC, vG, NULL, wsum, BC, BG, start, part, toC, adjC, &LC, &LG);
  free(toC);
  free(adjC);
  free(wsum);
  return OG_OK;
}

/* With fixed vertices the pre-check is on the split that keeps every free vertex on the GPU (the
 * CPU-pinned ones on the CPU); without, that split is all-GPU and its CPU load is 0. */
static int og_gggp_fix(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                       const int64_t* vC, const int64_t* vG, const int8_t* fix, int64_t BC, int64_t BG,
                       uint64_t seed, uint8_t* part, int32_t* trial_out) {
  int64_t LC0 = 0, LG0 = 0;
  for (int64_t v = 0; v < n; v++) {
    if (fix && fix[v] == 0)
      LC0 += vC[v];
    else
      LG0 += vG[v];
  }
  if ((LC0 <= BC && LG0 <= BG) || n == 0) {
    for (int64_t v = 0; v < n; v++) part[v] = (fix && fix[v] == 0) ? 0 : 1;
    *trial_out = -1;
    return OG_OK;
  }
  uint8_t* side = (uint8_t*)malloc((size_t)n);
  int64_t* toC = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  int64_t* adjC = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  int64_t* wsum = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!side || !toC || !adjC || !wsum) {
    free(side);
    free(toC);
    free(adjC);
    free(wsum);
    return OG_ERR_OOM;
  }
  for (int64_t v = 0; v < n; v++) {
    wsum[v] = 0;
    for (int64_t e = off[v]; e < off[v + 1]; e++) wsum[v] += W[e];
  }
  int best_t = -1, best_feas = 0;
  int64_t best_cut = 0;
  for (int t = 0; t < OG_TRIALS; t++) {
    const int64_t s = (int64_t)(og_hash(seed, 0xFFFFFFFFu, (uint32_t)t) % (uint64_t)n);
    int64_t LC, LG;
    const int64_t cut = og_grow(n, off, adj, W, vC, vG, fix, wsum, BC, BG, s, side, toC, adjC, &LC, &LG);
    const int feas = (LC <= BC && LG <= BG);
    if (best_t < 0 || feas > best_feas || (feas == best_feas && cut < best_cut)) {
      best_t = t;
      best_feas = feas;
      best_cut = cut;
      memcpy(part, side, (size_t)n);
    }
  }
  *trial_out = best_t;
  free(side);
  free(toC);
  free(adjC);
  free(wsum);
  return OG_OK;
}

int og_gggp(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W, const int64_t* vC,
            const int64_t* vG, int64_t BC, int64_t BG, uint64_t seed, uint8_t* part,
            int32_t* trial_out) {
  return og_gggp_fix(n, off, adj, W, vC, vG, NULL, BC, BG, seed, part, trial_out);
}

/* ------------------------------------------------------------------------ */
/* Refinement at one level: an optional balance round, then up to 8 gain     */
/* rounds.                                                                   */
/*                                                                           */
/* gain(v) = ext(v) - int(v): W to the other side minus W to its own side,    */
/* i.e. the cut decrease if v alone changes side.                             */
/*                                                                           */
/* Balance round (only when the split is infeasible).  The overloaded side s  */
/* is the one over its bound; if both are, the one with the larger relative   */
/* excess (L-B)/B, compared by cross-multiplication, CPU on ties.  All of s's */
/* vertices are ordered by (gain desc, id asc).  Take the shortest prefix     */
/* after whose move s is within its bound and the other side still within    */
/* its bound; if none exists, the longest prefix that keeps the other side    */
/* within its bound (possibly empty).                                        */
/*                                                                           */
/* Gain round r moves vertices from side r mod 2 to the other side.  Its      */
/* candidates are the source side's vertices with gain > 0, ordered by (gain  */
/* desc, id asc); the longest prefix whose added weight keeps the            */
/* destination within its bound moves, all at once.  Moves within one round  */
/* all go the same way, so the cut drops by at least the sum of their gains. */
/* Refinement stops after two consecutive rounds that move nothing.           */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t gain;
  int32_t id;
} og_cand;

static int og_cmp_cand(const void* a, const void* b) {
  const og_cand* x = (const og_cand*)a;
  const og_cand* y = (const og_cand*)b;
  if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;
  return (x->id > y->id) - (x->id < y->id);
}

static void og_gains(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                     const uint8_t* part, int64_t* gain) {
  for (int64_t v = 0; v < n; v++) {
    int64_t ext = 0, in = 0;
    for (int64_t e = off[v]; e < off[v + 1]; e++) {
      if (part[adj[e]] == part[v])
        in += W[e];
      else
        ext += W[e];
    }
    gain[v] = ext - in;
  }
}

/* Fixed vertices are never candidates, neither of the balance round nor of a gain round. */
static int og_refine_fix(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                         const int64_t* vC, const int64_t* vG, const int8_t* fix, int64_t BC,
                         int64_t BG, uint8_t* part, og_refine_stats* st) {
  int64_t* gain = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  og_cand* cand = (og_cand*)malloc((size_t)(n > 0 ? n : 1) * sizeof(og_cand));
  if (!gain || !cand) {
    free(gain);
    free(cand);
    return OG_ERR_OOM;
  }
  int64_t LC = 0, LG = 0;
  for (int64_t v = 0; v < n; v++) {
    if (part[v] == 0)
      LC += vC[v];
    else
      LG += vG[v];
  }
  memset(st, 0, sizeof(*st));

  if (!(LC <= BC && LG <= BG)) {
    const int overC = LC > BC, overG = LG > BG;
    int s;
    if (overC && overG) {
      const i128 lhs = (i128)(LC - BC) * (i128)BG;
      const i128 rhs = (i128)(LG - BG) * (i128)BC;
      s = (lhs >= rhs) ? 0 : 1;
    } else {
      s = overC ? 0 : 1;
    }
    og_gains(n, off, adj, W, part, gain);
    int64_t nc = 0;
    for (int64_t v = 0; v < n; v++)
      if (part[v] == s && !(fix && fix[v] >= 0)) {
        cand[nc].gain = gain[v];
        cand[nc].id = (int32_t)v;
        nc++;
      }
    qsort(cand, (size_t)nc, sizeof(og_cand), og_cmp_cand);
    const int64_t Ls = s == 0 ? LC : LG, Bs = s == 0 ? BC : BG;
    const int64_t Lo = s == 0 ? LG : LC, Bo = s == 0 ? BG : BC;
    const int64_t* cs = s == 0 ? vC : vG; /* weight leaving s   */
    const int64_t* co = s == 0 ? vG : vC; /* weight joining o   */
    int64_t k = -1, out_s = 0, in_o = 0;
    for (int64_t i = 0; i <= nc; i++) { /* prefix of length i */
      if (Ls - out_s <= Bs && Lo + in_o <= Bo) {
        k = i;
        break;
      }
      if (i < nc) {
        out_s += cs[cand[i].id];
        in_o += co[cand[i].id];
      }
    }
    if (k < 0) {
      k = 0;
      in_o = 0;
      for (int64_t i = 0; i <= nc; i++) {
        if (Lo + in_o <= Bo) k = i;
        if (i < nc) in_o += co[cand[i].id];
      }
    }
    for (int64_t i = 0; i < k; i++) {
      const int32_t v = cand[i].id;
      part[v] = (uint8_t)(1 - s);
      if (s == 0) {
        LC -= vC[v];
        LG += vG[v];
      } else {
        LG -= vG[v];
        LC += vC[v];
      }
    }
    st->balanced = 1;
    st->bal_moves = k;
  }

  int streak = 0;
  for (int r = 0; r < OG_REFINE_ROUNDS; r++) {
    const int src = r & 1, dst = 1 - src;
    og_gains(n, off, adj, W, part, gain);
    int64_t nc = 0;
    for (int64_t v = 0; v < n; v++)
      if (part[v] == src && gain[v] > 0 && !(fix && fix[v] >= 0)) {
        cand[nc].gain = gain[v];
        cand[nc].id = (int32_t)v;
        nc++;
      }
    qsort(cand, (size_t)nc, sizeof(og_cand), og_cmp_cand);
    const int64_t Ld = dst == 0 ? LC : LG, Bd = dst == 0 ? BC : BG;
    const int64_t* cd = dst == 0 ? vC : vG;
    int64_t k = 0, acc = 0;
    if (Ld <= Bd) {
      for (int64_t i = 0; i < nc; i++) {
        const int64_t c = cd[cand[i].id];
        if (acc + c > Bd - Ld) break;
        acc += c;
        k++;
      }
    }
    for (int64_t i = 0; i < k; i++) {
      const int32_t v = cand[i].id;
      part[v] = (uint8_t)dst;
      if (src == 0) {
        LC -= vC[v];
        LG += vG[v];
      } else {
        LG -= vG[v];
        LC += vC[v];
      }
    }
    st->rounds++;
    st->moves += k;
    streak = (k == 0) ? streak + 1 : 0;
    if (streak == 2) break;
  }
  st->load_cpu = LC;
  st->load_gpu = LG;
  free(gain);
  free(cand);
  return OG_OK;
}

int og_refine(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
              const int64_t* vC, const int64_t* vG, int64_t BC, int64_t BG, uint8_t* part,
              og_refine_stats* st) {
  return og_refine_fix(n, off, adj, W, vC, vG, NULL, BC, BG, part, st);
}

/* ------------------------------------------------------------------------ */
/* Cut of a split: sum of the transfer costs of directed edges whose ends are */
/* on different sides.                                                       */
/* ------------------------------------------------------------------------ */
int og_cut(int64_t n, const int64_t* off, const int32_t* cols, const int32_t* w,
           const uint8_t* part, int64_t* cut) {
  int64_t c = 0;
  for (int64_t u = 0; u < n; u++)
    for (int64_t e = off[u]; e < off[u + 1]; e++)
      if (part[u] != part[cols[e]]) c += w[e];
  *cut = c;
  return OG_OK;
}

static int64_t og_ucut(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* W,
                       const uint8_t* part) {
  int64_t c = 0;
  for (int64_t v = 0; v < n; v++)
    for (int64_t e = off[v]; e < off[v + 1]; e++)
      if (part[v] == 0 && part[adj[e]] == 1) c += W[e];
  return c;
}

/* ------------------------------------------------------------------------ */
/* The whole bipartitioner.                                                   */
/*                                                                           */
/*   B_C, B_G from Eq. (1)-(2) (or the given ratio) with the tolerance;       */
/*   level 0 = the symmetrised DAG with vertex weights (cC, cG);              */
/*   coarsen while the level has > 128 vertices and fewer than 48             */
/*   contractions were made: handshake rounds then two-hop pairing (caps     */
/*   B/8), and stop before contracting if the matching would keep more than  */
/*   95% of the vertices;                                                    */
/*   greedy graph growing on the coarsest level;                             */
/*   for each level from the coarsest to 0: project the coarser split (except */
/*   at the coarsest level), refine.                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t n, a;
  int64_t *off, *W, *vC, *vG;
  int32_t *adj, *cmap;
  int8_t* fix; /* NULL: no fixed vertices */
} og_level;

static void og_level_free(og_level* L) {
  free(L->off);
  free(L->W);
  free(L->vC);
  free(L->vG);
  free(L->adj);
  free(L->cmap);
  free(L->fix);
  memset(L, 0, sizeof(*L));
}

/* The multilevel bipartitioner.  fixed: NULL (all free), or one pin per vertex (-1 free, 0 CPU,
 * 1 GPU).  restrict_only = 0: the pins hold through every step (fixed vertices).  restrict_only = 1
 * (the V-cycle from a proposed split; every vertex carries its proposed side): the pins only keep
 * the matching to same-side pairs, the coarsest level's split is its pins, and refinement moves any
 * vertex. */
static int og_multilevel(int64_t n, int64_t m, const int64_t* off, const int32_t* cols,
                         const int32_t* w, const int32_t* cC, const int32_t* cG, const int8_t* fixed,
                         int restrict_only, double r_cpu, double tol, uint64_t seed, uint8_t* part,
                         og_result* res, og_trace* trace) {
  int st = og_validate(n, m, off, cols, w, cC, cG);
  if (st != OG_OK) return st;
  if (fixed)
    for (int64_t v = 0; v < n; v++)
      if (fixed[v] < -1 || fixed[v] > 1) return OG_ERR_INVALID;
  int64_t SC = 0, SG = 0;
  for (int64_t v = 0; v < n; v++) {
    SC += cC[v];
    SG += cG[v];
  }
  int64_t BC, BG;
  st = og_bounds(SC, SG, r_cpu, tol, &BC, &BG);
  if (st != OG_OK) return st;
  memset(res, 0, sizeof(*res));
  if (trace) memset(trace, 0, sizeof(*trace));
  res->bound_cpu = BC;
  res->bound_gpu = BG;
  if (n == 0) {
    res->feasible = 1;
    if (trace) trace->gggp_trial = -1;
    return OG_OK;
  }

  og_level lv[OG_MAX_LEVELS + 1];
  memset(lv, 0, sizeof(lv));
  int rc = OG_ERR_OOM;
  uint8_t* pc = NULL;
  uint8_t* pf = NULL;
  lv[0].n = n;
  lv[0].off = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
  lv[0].adj = (int32_t*)malloc((size_t)(2 * m + 1) * sizeof(int32_t));
  lv[0].W = (int64_t*)malloc((size_t)(2 * m + 1) * sizeof(int64_t));
  lv[0].vC = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  lv[0].vG = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!lv[0].off || !lv[0].adj || !lv[0].W || !lv[0].vC || !lv[0].vG) goto done;
  for (int64_t v = 0; v < n; v++) {
    lv[0].vC[v] = cC[v];
    lv[0].vG[v] = cG[v];
  }
  if (fixed) {
    lv[0].fix = (int8_t*)malloc((size_t)n);
    if (!lv[0].fix) goto done;
    memcpy(lv[0].fix, fixed, (size_t)n);
  }
  st = og_symmetrize(n, m, off, cols, w, lv[0].off, lv[0].adj, lv[0].W, &lv[0].a);
  if (st != OG_OK) {
    rc = st;
    goto done;
  }

  /* coarsening */
  int L = 0;
  const int64_t capC = BC / OG_CAP_DIV, capG = BG / OG_CAP_DIV;
  while (lv[L].n > OG_COARSEST && L < OG_MAX_LEVELS) {
    og_level* f = &lv[L];
    int32_t* mate = (int32_t*)malloc((size_t)f->n * sizeof(int32_t));
    if (!mate) goto done;
    if (og_match_fix(f->n, f->off, f->adj, f->W, f->vC, f->vG, f->fix, capC, capG, seed,
                     OG_MATCH_ROUNDS, mate) != OG_OK ||
        og_match_twohop_fix(f->n, f->off, f->adj, f->W, f->vC, f->vG, f->fix, capC, capG, seed,
                            mate) != OG_OK) {
      free(mate);
      goto done;
    }
    const int64_t nc = og_count_coarse(f->n, mate);
    if (nc * OG_STALL_DEN > f->n * OG_STALL_NUM) {
      free(mate);
      break;
    }
    og_level* c = &lv[L + 1];
    f->cmap = (int32_t*)malloc((size_t)f->n * sizeof(int32_t));
    c->off = (int64_t*)malloc((size_t)(nc + 1) * sizeof(int64_t));
    c->adj = (int32_t*)malloc((size_t)(f->a + 1) * sizeof(int32_t));
    c->W = (int64_t*)malloc((size_t)(f->a + 1) * sizeof(int64_t));
    c->vC = (int64_t*)malloc((size_t)nc * sizeof(int64_t));
    c->vG = (int64_t*)malloc((size_t)nc * sizeof(int64_t));
    if (!f->cmap || !c->off || !c->adj || !c->W || !c->vC || !c->vG) {
      free(mate);
      goto done;
    }
    st = og_contract(f->n, f->off, f->adj, f->W, f->vC, f->vG, mate, f->cmap, &c->n, c->off,
                     c->adj, c->W, c->vC, c->vG, &c->a);
    free(mate);
    if (st != OG_OK) goto done;
    if (f->fix) { /* a coarse vertex is pinned where a member is (members are compatible) */
      c->fix = (int8_t*)malloc((size_t)(nc > 0 ? nc : 1));
      if (!c->fix) goto done;
      for (int64_t x = 0; x < nc; x++) c->fix[x] = -1;
      for (int64_t v = 0; v < f->n; v++)
        if (f->fix[v] > c->fix[f->cmap[v]]) c->fix[f->cmap[v]] = f->fix[v];
    }
    L++;
  }

  /* initial split on the coarsest level */
  pc = (uint8_t*)malloc((size_t)lv[L].n);
  if (!pc) goto done;
  int32_t trial = -1;
  if (restrict_only) { /* every coarse vertex holds members of one proposed side */
    for (int64_t x = 0; x < lv[L].n; x++) pc[x] = (uint8_t)lv[L].fix[x];
  } else if (og_gggp_fix(lv[L].n, lv[L].off, lv[L].adj, lv[L].W, lv[L].vC, lv[L].vG, lv[L].fix, BC, BG,
                         seed, pc, &trial) != OG_OK) {
    goto done;
  }

  /* uncoarsening */
  int32_t rounds_total = 0;
  og_refine_stats rs;
  memset(&rs, 0, sizeof(rs));
  for (int l = L; l >= 0; l--) {
    if (l < L) {
      pf = (uint8_t*)malloc((size_t)lv[l].n);
      if (!pf) goto done;
      for (int64_t v = 0; v < lv[l].n; v++) pf[v] = pc[lv[l].cmap[v]];
      free(pc);
      pc = pf;
      pf = NULL;
    }
    if (og_refine_fix(lv[l].n, lv[l].off, lv[l].adj, lv[l].W, lv[l].vC, lv[l].vG,
                      restrict_only ? NULL : lv[l].fix, BC, BG, pc, &rs) != OG_OK)
      goto done;
    rounds_total += rs.rounds;
    if (trace) {
      trace->rounds[l] = rs.rounds;
      trace->moves[l] = rs.moves;
      trace->balanced[l] = rs.balanced;
      trace->bal_moves[l] = rs.bal_moves;
      trace->cut[l] = og_ucut(lv[l].n, lv[l].off, lv[l].adj, lv[l].W, pc);
    }
  }
  memcpy(part, pc, (size_t)n);
  og_cut(n, off, cols, w, part, &res->cut);
  res->load_cpu = rs.load_cpu;
  res->load_gpu = rs.load_gpu;
  res->feasible = (rs.load_cpu <= BC && rs.load_gpu <= BG);
  res->levels = L;
  res->rounds = rounds_total;
  res->coarsest_n = (int32_t)lv[L].n;
  if (trace) {
    trace->levels = L;
    trace->gggp_trial = trial;
    for (int l = 0; l <= L; l++) {
      trace->n[l] = lv[l].n;
      trace->a[l] = lv[l].a;
    }
  }
  rc = OG_OK;
done:
  free(pc);
  free(pf);
  for (int l = 0; l <= OG_MAX_LEVELS; l++) og_level_free(&lv[l]);
  return rc;
}

int og_partition_fixed(int64_t n, int64_t m, const int64_t* off, const int32_t* cols,
                       const int32_t* w, const int32_t* cC, const int32_t* cG, const int8_t* fixed,
                       double r_cpu, double tol, uint64_t seed, uint8_t* part, og_result* res,
                       og_trace* trace) {
  return og_multilevel(n, m, off, cols, w, cC, cG, fixed, 0, r_cpu, tol, seed, part, res, trace);
}

int og_partition(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                 const int32_t* cC, const int32_t* cG, double r_cpu, double tol, uint64_t seed,
                 uint8_t* part, og_result* res, og_trace* trace) {
  return og_partition_fixed(n, m, off, cols, w, cC, cG, NULL, r_cpu, tol, seed, part, res, trace);
}

/* ------------------------------------------------------------------------ */
/* Topological levels: level(v) = 0 for a vertex without predecessors, else   */
/* 1 + the largest level of its predecessors.                                 */
/* ------------------------------------------------------------------------ */
int og_levels(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, int32_t* level,
              int32_t* nlevels) {
  (void)m;
  int64_t* indeg = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!indeg || !queue) {
    free(indeg);
    free(queue);
    return OG_ERR_OOM;
  }
  for (int64_t e = 0; e < off[n]; e++) indeg[cols[e]]++;
  int64_t head = 0, tail = 0;
  for (int64_t v = 0; v < n; v++) {
    level[v] = 0;
    if (indeg[v] == 0) queue[tail++] = (int32_t)v;
  }
  int32_t maxl = -1;
  while (head < tail) {
    const int32_t v = queue[head++];
    if (level[v] > maxl) maxl = level[v];
    for (int64_t e = off[v]; e < off[v + 1]; e++) {
      const int32_t u = cols[e];
      if (level[v] + 1 > level[u]) level[u] = level[v] + 1;
      if (--indeg[u] == 0) queue[tail++] = u;
    }
  }
  free(indeg);
  free(queue);
  if (tail != n) return OG_ERR_NOT_DAG;
  *nlevels = maxl + 1;
  return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* Makespan of a mapping with as many workers as needed on each side:         */
/*   finish(v) = t_part(v)(v) + max over u->v of (finish(u) + w(u,v) if u and */
/*               v sit on different sides, else finish(u)),  max of none = 0; */
/*   makespan  = max over v of finish(v)  (0 for an empty graph).            */
/* Vertices are taken in a topological order (Kahn's algorithm).             */
/* ------------------------------------------------------------------------ */
int og_makespan(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                const int32_t* cC, const int32_t* cG, const uint8_t* part, int64_t* finish,
                int64_t* makespan) {
  int st = og_validate(n, m, off, cols, w, cC, cG);
  if (st != OG_OK) return st;
  for (int64_t v = 0; v < n; v++)
    if (part[v] > 1) return OG_ERR_INVALID;
  int64_t* indeg = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int64_t* start = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int64_t* fin = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!indeg || !start || !fin || !queue) {
    free(indeg);
    free(start);
    free(fin);
    free(queue);
    return OG_ERR_OOM;
  }
  for (int64_t e = 0; e < m; e++) indeg[cols[e]]++;
  int64_t head = 0, tail = 0;
  for (int64_t v = 0; v < n; v++)
    if (indeg[v] == 0) queue[tail++] = (int32_t)v;
  int64_t ms = 0;
  while (head < tail) {
    const int32_t v = queue[head++];
    fin[v] = start[v] + (part[v] ? cG[v] : cC[v]);
    if (fin[v] > ms) ms = fin[v];
    for (int64_t e = off[v]; e < off[v + 1]; e++) {
      const int32_t u = cols[e];
      const int64_t t = fin[v] + (part[u] != part[v] ? w[e] : 0);
      if (t > start[u]) start[u] = t;
      if (--indeg[u] == 0) queue[tail++] = u;
    }
  }
  if (finish)
    for (int64_t v = 0; v < n; v++) finish[v] = fin[v];
  *makespan = ms;
  free(indeg);
  free(start);
  free(fin);
  free(queue);
  return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* Learned proposal: order, then split.                                       */
/*                                                                           */
/* A logit's sort key is its IEEE-754 bit pattern mapped to an unsigned      */
/* integer that increases with the float's total order (negative values:     */
/* all bits flipped; others: sign bit set).  Vertices are visited by         */
/* decreasing key, smaller id first on equal keys; visiting one moves it      */
/* from the GPU side to the CPU side.  k = min(kC, kG) with kC the largest    */
/* prefix length whose CPU load stays within B_C and kG the smallest prefix   */
/* length whose remaining GPU load is within B_G.                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t key;
  int32_t id;
} og_lkey;

static uint32_t og_float_key(float f) {
  uint32_t b;
  memcpy(&b, &f, sizeof(b));
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

static int og_cmp_lkey(const void* a, const void* b) {
  const og_lkey* x = (const og_lkey*)a;
  const og_lkey* y = (const og_lkey*)b;
  if (x->key != y->key) return x->key > y->key ? -1 : 1; /* larger logit first */
  return (x->id > y->id) - (x->id < y->id);
}

int og_propose(int64_t n, const float* logits, const int64_t* vC, const int64_t* vG, int64_t BC,
               int64_t BG, uint8_t* part, int64_t* k_out) {
  for (int64_t v = 0; v < n; v++)
    if (isnan(logits[v])) return OG_ERR_INVALID;
  og_lkey* order = (og_lkey*)malloc((size_t)(n > 0 ? n : 1) * sizeof(og_lkey));
  if (!order) return OG_ERR_OOM;
  int64_t SG = 0;
  for (int64_t v = 0; v < n; v++) {
    order[v].key = og_float_key(logits[v]);
    order[v].id = (int32_t)v;
    SG += vG[v];
  }
  qsort(order, (size_t)n, sizeof(og_lkey), og_cmp_lkey);
  /* kC: largest k with sum of the first k CPU costs <= B_C */
  int64_t kC = 0, LC = 0;
  while (kC < n && LC + vC[order[kC].id] <= BC) {
    LC += vC[order[kC].id];
    kC++;
  }
  /* kG: smallest k with SG - sum of the first k GPU costs <= B_G */
  int64_t kG = 0, LG = SG;
  while (kG < n && LG > BG) {
    LG -= vG[order[kG].id];
    kG++;
  }
  const int64_t k = kC < kG ? kC : kG;
  for (int64_t v = 0; v < n; v++) part[v] = 1;
  for (int64_t i = 0; i < k; i++) part[order[i].id] = 0;
  if (k_out) *k_out = k;
  free(order);
  return OG_OK;
}

int og_partition_learned(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                         const int32_t* cC, const int32_t* cG, const float* logits, double r_cpu,
                         double tol, uint8_t* part, og_result* res) {
  int st = og_validate(n, m, off, cols, w, cC, cG);
  if (st != OG_OK) return st;
  int64_t SC = 0, SG = 0;
  for (int64_t v = 0; v < n; v++) {
    SC += cC[v];
    SG += cG[v];
  }
  int64_t BC, BG;
  st = og_bounds(SC, SG, r_cpu, tol, &BC, &BG);
  if (st != OG_OK) return st;
  memset(res, 0, sizeof(*res));
  res->bound_cpu = BC;
  res->bound_gpu = BG;
  if (n == 0) {
    res->feasible = 1;
    return OG_OK;
  }
  int64_t* uoff = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
  int32_t* uadj = (int32_t*)malloc((size_t)(2 * m + 1) * sizeof(int32_t));
  int64_t* uW = (int64_t*)malloc((size_t)(2 * m + 1) * sizeof(int64_t));
  int64_t* vC = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  int64_t* vG = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  int rc = OG_ERR_OOM;
  if (!uoff || !uadj || !uW || !vC || !vG) goto done;
  for (int64_t v = 0; v < n; v++) {
    vC[v] = cC[v];
    vG[v] = cG[v];
  }
  int64_t a = 0;
  st = og_symmetrize(n, m, off, cols, w, uoff, uadj, uW, &a);
  if (st != OG_OK) {
    rc = st;
    goto done;
  }
  st = og_propose(n, logits, vC, vG, BC, BG, part, NULL);
  if (st != OG_OK) {
    rc = st;
    goto done;
  }
  og_refine_stats rs;
  st = og_refine(n, uoff, uadj, uW, vC, vG, BC, BG, part, &rs);
  if (st != OG_OK) {
    rc = st;
    goto done;
  }
  og_cut(n, off, cols, w, part, &res->cut);
  res->load_cpu = rs.load_cpu;
  res->load_gpu = rs.load_gpu;
  res->feasible = (rs.load_cpu <= BC && rs.load_gpu <= BG);
  res->levels = 0;
  res->rounds = rs.rounds;
  res->coarsest_n = (int32_t)n;
  rc = OG_OK;
done:
  free(uoff);
  free(uadj);
  free(uW);
  free(vC);
  free(vG);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Makespan of a mapping on a fixed number of workers per side (the testbed   */
/* of Sec. IV.A runs kernels on 3 CPU worker cores and 1 GPU worker): a list  */
/* schedule, simulated event by event in time order.                          */
/*                                                                           */
/*   - A task v runs without preemption on one worker of side part[v] for    */
/*     its cost on that side; each side has its own workers (P_C, P_G).      */
/*   - Its data are there at r(v) = max over in-entries u->v of finish(u),   */
/*     plus w(u,v) when u sits on the other side (every parallel entry is a  */
/*     transfer of its own; transfers do not compete); r = 0 for a source.   */
/*   - At each time t, in increasing order: first every running task that    */
/*     ends at or before t ends (its worker becomes idle, and each successor */
/*     whose last predecessor this was is released); then, on each side,     */
/*     while a worker is idle and a released task with r <= t waits, the     */
/*     waiting task with the smallest (r, id) starts at t.  t then moves to  */
/*     the next end of a running task or, on a side with an idle worker, to  */
/*     the smallest r among its waiting tasks, whichever comes first.        */
/*   - makespan = the largest finish time (0 for an empty graph).            */
/* Identical idle workers are interchangeable, so the times do not depend on */
/* which idle worker takes a task.  With at least n workers on both sides    */
/* every task starts at r(v) and the result is og_makespan's.                */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t t;  /* ready time (waiting heaps) or end time (running heap) */
  int32_t v;
} og_ev;

static int og_ev_less(const og_ev* a, const og_ev* b) {
  return a->t < b->t || (a->t == b->t && a->v < b->v);
}

static void og_heap_push(og_ev* h, int64_t* len, og_ev x) {
  int64_t i = (*len)++;
  while (i > 0) {
    const int64_t p = (i - 1) / 2;
    if (!og_ev_less(&x, &h[p])) break;
    h[i] = h[p];
    i = p;
  }
  h[i] = x;
}

static og_ev og_heap_pop(og_ev* h, int64_t* len) {
  const og_ev top = h[0];
  const og_ev x = h[--(*len)];
  int64_t i = 0;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= *len) break;
    if (c + 1 < *len && og_ev_less(&h[c + 1], &h[c])) c++;
    if (!og_ev_less(&h[c], &x)) break;
    h[i] = h[c];
    i = c;
  }
  if (*len > 0) h[i] = x;
  return top;
}

int og_makespan_workers(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                        const int32_t* cC, const int32_t* cG, const uint8_t* part, int64_t workers_cpu,
                        int64_t workers_gpu, int64_t* finish, int64_t* makespan) {
  int st = og_validate(n, m, off, cols, w, cC, cG);
  if (st != OG_OK) return st;
  if (workers_cpu < 1 || workers_gpu < 1) return OG_ERR_INVALID;
  for (int64_t v = 0; v < n; v++)
    if (part[v] > 1) return OG_ERR_INVALID;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  int64_t* pending = (int64_t*)calloc(nn, sizeof(int64_t));
  int64_t* ready = (int64_t*)calloc(nn, sizeof(int64_t));
  int64_t* fin = (int64_t*)calloc(nn, sizeof(int64_t));
  og_ev* wait[2] = {(og_ev*)malloc(nn * sizeof(og_ev)), (og_ev*)malloc(nn * sizeof(og_ev))};
  og_ev* run = (og_ev*)malloc(nn * sizeof(og_ev));
  if (!pending || !ready || !fin || !wait[0] || !wait[1] || !run) {
    free(pending);
    free(ready);
    free(fin);
    free(wait[0]);
    free(wait[1]);
    free(run);
    return OG_ERR_OOM;
  }
  for (int64_t e = 0; e < m; e++) pending[cols[e]]++;
  int64_t wlen[2] = {0, 0}, rlen = 0;
  int64_t idle[2] = {workers_cpu, workers_gpu};
  for (int64_t v = 0; v < n; v++)
    if (pending[v] == 0) {
      og_ev x = {0, (int32_t)v};
      og_heap_push(wait[part[v]], &wlen[part[v]], x);
    }
  int64_t t = 0, ms = 0;
  for (;;) {
    /* ends at or before t */
    while (rlen > 0 && run[0].t <= t) {
      const og_ev done = og_heap_pop(run, &rlen);
      const int32_t u = done.v;
      idle[part[u]]++;
      for (int64_t e = off[u]; e < off[u + 1]; e++) {
        const int32_t v = cols[e];
        const int64_t arrive = fin[u] + (part[u] != part[v] ? w[e] : 0);
        if (arrive > ready[v]) ready[v] = arrive;
        if (--pending[v] == 0) {
          og_ev x = {ready[v], v};
          og_heap_push(wait[part[v]], &wlen[part[v]], x);
        }
      }
    }
    /* starts at t */
    for (int s = 0; s < 2; s++)
      while (idle[s] > 0 && wlen[s] > 0 && wait[s][0].t <= t) {
        const og_ev x = og_heap_pop(wait[s], &wlen[s]);
        const int32_t v = x.v;
        fin[v] = t + (part[v] ? cG[v] : cC[v]);
        if (fin[v] > ms) ms = fin[v];
        og_ev r = {fin[v], v};
        og_heap_push(run, &rlen, r);
        idle[s]--;
      }
    if (rlen > 0 && run[0].t <= t) continue; /* a task of cost 0 ended at t */
    int64_t next = INT64_MAX;
    if (rlen > 0) next = run[0].t;
    for (int s = 0; s < 2; s++)
      if (idle[s] > 0 && wlen[s] > 0 && wait[s][0].t < next) next = wait[s][0].t;
    if (next == INT64_MAX) break;
    t = next;
  }
  if (finish)
    for (int64_t v = 0; v < n; v++) finish[v] = fin[v];
  *makespan = ms;
  free(pending);
  free(ready);
  free(fin);
  free(wait[0]);
  free(wait[1]);
  free(run);
  return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* The learned path as a V-cycle: the proposal from the logits (og_propose)  */
/* gives every vertex a side; coarsening matches only vertices proposed to   */
/* the same side (the proposal's sides are pins for the matching and the     */
/* two-hop pairing only), so every coarse vertex has one proposed side, and  */
/* the coarsest level's split is those sides; then every level is refined    */
/* on the way back up exactly as in og_partition (projection, balance round, */
/* gain rounds, with every vertex free to move).                             */
/* ------------------------------------------------------------------------ */
int og_partition_vcycle(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                        const int32_t* cC, const int32_t* cG, const float* logits, double r_cpu,
                        double tol, uint64_t seed, uint8_t* part, og_result* res, og_trace* trace) {
  int st = og_validate(n, m, off, cols, w, cC, cG);
  if (st != OG_OK) return st;
  int64_t SC = 0, SG = 0;
  for (int64_t v = 0; v < n; v++) {
    SC += cC[v];
    SG += cG[v];
  }
  int64_t BC, BG;
  st = og_bounds(SC, SG, r_cpu, tol, &BC, &BG);
  if (st != OG_OK) return st;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  int64_t* vC = (int64_t*)malloc(nn * sizeof(int64_t));
  int64_t* vG = (int64_t*)malloc(nn * sizeof(int64_t));
  uint8_t* prop = (uint8_t*)malloc(nn);
  int8_t* pin = (int8_t*)malloc(nn);
  int rc = OG_ERR_OOM;
  if (!vC || !vG || !prop || !pin) goto done;
  for (int64_t v = 0; v < n; v++) {
    vC[v] = cC[v];
    vG[v] = cG[v];
  }
  rc = og_propose(n, logits, vC, vG, BC, BG, prop, NULL);
  if (rc != OG_OK) goto done;
  for (int64_t v = 0; v < n; v++) pin[v] = (int8_t)prop[v];
  rc = og_multilevel(n, m, off, cols, w, cC, cG, pin, 1, r_cpu, tol, seed, part, res, trace);
done:
  free(vC);
  free(vG);
  free(prop);
  free(pin);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* k device classes by recursive bisection (Sec. VI names a third kind of    */
/* processor, an FPGA, as future work; this is the project's reading).        */
/*                                                                           */
/*   - costs[i * n + v] is v's time on class i (int32, >= 0); a transfer     */
/*     between any two different classes costs w(e).                         */
/*   - Two groups of classes act as two devices: a group's time for v is the */
/*     classes' times combined like parallel resistors, folded left to       */
/*     right with comb(x, y) = floor(x*y / (x+y)) (0 when x + y = 0); for    */
/*     one class it is that class's time.  (k = 2 is then the 2-way problem  */
/*     with c_CPU = costs[0], c_GPU = costs[1].)                             */
/*   - bisect(V', [lo, hi)): one class left -> every vertex of V' gets it.   */
/*     Otherwise mid = lo + ceil((hi - lo) / 2); the subgraph induced by V'  */
/*     (vertices renumbered in increasing id, every entry with both ends in  */
/*     V' kept) is split by og_partition with cpu_cost = the group time of   */
/*     [lo, mid), gpu_cost = that of [mid, hi), the bounds of Eq. (1) from   */
/*     their sums, tolerance tol and `seed`; side 0 recurses into [lo, mid), */
/*     side 1 into [mid, hi).  An empty side ends its branch.                */
/*   - Outputs: cls[v]; the cut (sum of w over directed entries whose ends   */
/*     have different classes); loads[i] = sum of costs[i][v] over class-i   */
/*     vertices; feasible = every bisection was feasible; the number of      */
/*     bisections run.                                                       */
/* ------------------------------------------------------------------------ */
static int64_t og_comb(int64_t x, int64_t y) {
  if (x + y == 0) return 0;
  return (int64_t)(((__int128)x * (__int128)y) / (__int128)(x + y));
}

static int og_bisect(int64_t n, const int64_t* off, const int32_t* cols, const int32_t* w, int64_t n_all,
                     const int32_t* costs, const int32_t* orig, int lo, int hi, double tol, uint64_t seed,
                     uint8_t* cls, int32_t* feasible, int32_t* count) {
  if (n == 0) return OG_OK;
  if (hi - lo == 1) {
    for (int64_t v = 0; v < n; v++) cls[orig[v]] = (uint8_t)lo;
    return OG_OK;
  }
  const int mid = lo + (hi - lo + 1) / 2;
  const size_t nn = (size_t)n;
  int32_t* cA = (int32_t*)malloc(nn * sizeof(int32_t));
  int32_t* cB = (int32_t*)malloc(nn * sizeof(int32_t));
  uint8_t* part = (uint8_t*)malloc(nn);
  int rc = OG_ERR_OOM;
  int64_t* soff = NULL;
  int32_t *scols = NULL, *sw = NULL, *sorig = NULL, *newid = NULL;
  if (!cA || !cB || !part) goto done;
  for (int64_t v = 0; v < n; v++) {
    int64_t a = costs[(int64_t)lo * n_all + orig[v]];
    for (int c = lo + 1; c < mid; c++) a = og_comb(a, costs[(int64_t)c * n_all + orig[v]]);
    int64_t b = costs[(int64_t)mid * n_all + orig[v]];
    for (int c = mid + 1; c < hi; c++) b = og_comb(b, costs[(int64_t)c * n_all + orig[v]]);
    cA[v] = (int32_t)a;
    cB[v] = (int32_t)b;
  }
  og_result res;
  rc = og_partition(n, off[n], off, cols, w, cA, cB, -1.0, tol, seed, part, &res, NULL);
  if (rc != OG_OK) goto done;
  (*count)++;
  if (!res.feasible) *feasible = 0;
  newid = (int32_t*)malloc(nn * sizeof(int32_t));
  soff = (int64_t*)malloc((nn + 1) * sizeof(int64_t));
  scols = (int32_t*)malloc((size_t)(off[n] > 0 ? off[n] : 1) * sizeof(int32_t));
  sw = (int32_t*)malloc((size_t)(off[n] > 0 ? off[n] : 1) * sizeof(int32_t));
  sorig = (int32_t*)malloc(nn * sizeof(int32_t));
  rc = OG_ERR_OOM;
  if (!newid || !soff || !scols || !sw || !sorig) goto done;
  for (int side = 0; side < 2; side++) {
    int64_t sn = 0;
    for (int64_t v = 0; v < n; v++) newid[v] = part[v] == side ? (int32_t)sn++ : -1;
    int64_t se = 0;
    soff[0] = 0;
    for (int64_t v = 0; v < n; v++) {
      if (part[v] != side) continue;
      sorig[newid[v]] = orig[v];
      for (int64_t e = off[v]; e < off[v + 1]; e++)
        if (part[cols[e]] == side) {
          scols[se] = newid[cols[e]];
          sw[se] = w[e];
          se++;
        }
      soff[newid[v] + 1] = se;
    }
    rc = og_bisect(sn, soff, scols, sw, n_all, costs, sorig, side ? mid : lo, side ? hi : mid, tol, seed, cls,
                   feasible, count);
    if (rc != OG_OK) goto done;
  }
  rc = OG_OK;
done:
  free(cA);
  free(cB);
  free(part);
  free(newid);
  free(soff);
  free(scols);
  free(sw);
  free(sorig);
  return rc;
}

int og_partition_kway(int64_t n, int64_t m, const int64_t* off, const int32_t* cols, const int32_t* w,
                      int32_t k, const int32_t* costs, double tol, uint64_t seed, uint8_t* cls, int64_t* cut,
                      int64_t* loads, int32_t* feasible, int32_t* bisections) {
  /* checks in the precedence of og_validate: INVALID (arguments, any class's negative time, the
   * CSR), then OVERFLOW (a class's or the transfers' sum above 2^61), then NOT_DAG */
  if (k < 1 || k > 255 || n < 0 || !(tol >= 0.0 && tol <= 1.0)) return OG_ERR_INVALID;
  for (int64_t i = 0; i < (int64_t)k * n; i++)
    if (costs[i] < 0) return OG_ERR_INVALID;
  const int st0 = og_validate(n, m, off, cols, w, costs, costs);
  if (st0 == OG_ERR_INVALID) return st0;
  for (int32_t i = 0; i < k; i++) {
    int64_t s = 0;
    for (int64_t v = 0; v < n; v++) s += costs[(int64_t)i * n + v];
    if (s > OG_SUM_LIMIT) return OG_ERR_OVERFLOW;
  }
  if (st0 != OG_OK) return st0;
  int32_t* orig = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  if (!orig) return OG_ERR_OOM;
  for (int64_t v = 0; v < n; v++) orig[v] = (int32_t)v;
  *feasible = 1;
  *bisections = 0;
  const int rc = og_bisect(n, off, cols, w, n, costs, orig, 0, k, tol, seed, cls, feasible, bisections);
  free(orig);
  if (rc != OG_OK) return rc;
  int64_t c = 0;
  for (int64_t u = 0; u < n; u++)
    for (int64_t e = off[u]; e < off[u + 1]; e++)
      if (cls[u] != cls[cols[e]]) c += w[e];
  *cut = c;
  for (int32_t i = 0; i < k; i++) loads[i] = 0;
  for (int64_t v = 0; v < n; v++) loads[cls[v]] += costs[(int64_t)cls[v] * n + v];
  return OG_OK;
}
