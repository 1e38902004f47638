/*
 * rpForests CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-sequential C restatement of random projection
 * forests kNN search (Yan, Wang, Wang, Wang, Li, "K-nearest Neighbor Search
 * by Random Projection Forests", arXiv 1812.11689).  Only tests/, the smoke
 * check of __graft_entry__ and the cpu_baseline leg of bench.py may load it.
 * It shares no source with the CUDA library and includes none of its headers.
 *
 * What it computes, step by step, in the paper's order:
 *   rpTree growth          -- Sec. 2, Algorithm 1 (rpTree(U))
 *   direction choice       -- Sec. 2, Algorithm 2 (whichProjection(W, nTry))
 *   ensemble kNN search    -- Sec. 2, Algorithm 3 (kNNrpForests(Q, U))
 *   exact brute-force kNN  -- ground truth for the Sec. 5.1 metrics
 *
 * Readings of points where the paper is silent (each restated where used):
 *   leaf rule   : a node with more than L points is split, so no leaf holds
 *                 more than L points (the leaf size bound of Sec. 5.2; the
 *                 n_s of Algorithm 1 is L + 1).
 *   randomness  : every random draw is a pure function of (seed, tree, node
 *                 key, ...) through a SplitMix64 chain, so the order in which
 *                 Algorithm 1 picks nodes from its working set is irrelevant.
 *   direction   : r = g * (1 / |g|), g ~ N(0, I_d) by FP32 Box-Muller on our
 *                 own FP32 ln and sin/cos series (no libm transcendental);
 *                 |g| and r in FP32 (r stored as doubles).
 *   projection  : p = fold_k fma((double)x_k, r_k, p) from +0.0 (FP64).
 *   dispersion  : V = canonical-order sum of (p - mu)^2 with mu = S / m and
 *                 S the canonical-order sum of p (argmax of V == argmax SD).
 *   split point : c = fma(u, b - a, a), u uniform in [0,1); accepted iff
 *                 a < c <= b, else redrawn (8 attempts), else a rank split.
 *                 Median rule: the floor(m/2) points smallest in
 *                 (projection, point index) order go left; c = the
 *                 projection of the first point that goes right.
 *   distance    : d32 = fold_k fmaf(x_k - y_k, x_k - y_k, s) in FP32, ties
 *                 broken by the smaller index; reported distance sqrtf(d32).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-math-errno -fopenmp -fPIC
 * -shared.  -ffp-contract=off is essential: every fused multiply-add here is
 * written explicitly with fma()/fmaf(), and nothing else may be fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_GAMMA 0x9E3779B97F4A7C15ULL
#define ORC_TAG_DIR 1ULL
#define ORC_TAG_SPLIT 2ULL
#define ORC_SPLIT_ATTEMPTS 8
#define ORC_CHUNK 4096

/* ------------------------------------------------------------------------- */
/* Counter-based random numbers.  mix64 is the SplitMix64 output function    */
/* (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",   */
/* OOPSLA 2014); the SplitMix64 sequence for state s is mix64(s + i*GAMMA).   */
/* ------------------------------------------------------------------------- */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* word(seed, tag, t, key, j, c): absorb the five fields in this order. */
uint64_t orc_word(uint64_t seed, uint64_t tag, uint64_t t, uint64_t key,
                  uint64_t j, uint64_t c) {
  uint64_t f[5] = {tag, t, key, j, c};
  uint64_t h = seed;
  for (int i = 0; i < 5; ++i) h = orc_mix64((h ^ f[i]) + ORC_GAMMA);
  return h;
}

/* Child node keys: root key 1; side 0 = left child, 1 = right child. */
uint64_t orc_child_key(uint64_t key, int side) {
  return orc_mix64(key ^ ((uint64_t)(1 + side) * ORC_GAMMA));
}

/* u53 in [0, 1). */
double orc_u53(uint64_t w) { return (double)(w >> 11) * 0x1p-53; }

/* ------------------------------------------------------------------------- */
/* Natural logarithm in FP32 for normal u > 0: u = m 2^e with m folded into   */
/* [sqrt(2)/2, sqrt(2)], ln m = 2 atanh(s), s = (m-1)/(m+1), and the atanh    */
/* Taylor series s (1 + z/3 + z^2/5 + ... + z^5/11), z = s^2 <= 0.0295.       */
/* Coefficients are the FP32 roundings of the double quotients 1/(2k+1).      */
/* ------------------------------------------------------------------------- */
static const float ORC_LN2F = 0.693147180559945309f;
static const float ORC_SQRT2F = 1.41421356237309504f;
#define ORC_LN_TERMS 6 /* k = 0..5 */

float orc_lnf(float u) {
  uint32_t b;
  memcpy(&b, &u, 4);
  int e = (int)((b >> 23) & 0xff) - 127;
  uint32_t mb = (b & 0x007FFFFFu) | 0x3F800000u;
  float m;
  memcpy(&m, &mb, 4);
  if (m > ORC_SQRT2F) {
    m = m * 0.5f;
    e += 1;
  }
  float s = (m - 1.0f) / (m + 1.0f);
  float z = s * s;
  float p = (float)(1.0 / (double)(2 * (ORC_LN_TERMS - 1) + 1));
  for (int k = ORC_LN_TERMS - 2; k >= 0; --k) p = fmaf(p, z, (float)(1.0 / (double)(2 * k + 1)));
  float h = s * p;
  return fmaf((float)e, ORC_LN2F, h + h);
}

/* ------------------------------------------------------------------------- */
/* cos(2 pi u) and sin(2 pi u) in FP32 for u in [0, 1): quadrant q =          */
/* floor(4u), theta = (4u - q) pi/2 in [0, pi/2), Taylor series of cos and    */
/* sin to theta^12 and theta^13 (7 terms each).  Coefficients (-1)^k / n! are */
/* the FP32 roundings of 1 / (running double product n!).                    */
/* ------------------------------------------------------------------------- */
static const float ORC_PI_2F = 1.57079632679489662f;
#define ORC_TRIG_TERMS 7

static void orc_trig_coefs(float* cosc, float* sinc) {
  double inv[2 * ORC_TRIG_TERMS];
  double fact = 1.0;
  inv[0] = 1.0;
  for (int n = 1; n <= 2 * ORC_TRIG_TERMS - 1; ++n) {
    fact = fact * (double)n;
    inv[n] = 1.0 / fact;
  }
  for (int k = 0; k < ORC_TRIG_TERMS; ++k) {
    cosc[k] = (float)((k & 1) ? -inv[2 * k] : inv[2 * k]);
    sinc[k] = (float)((k & 1) ? -inv[2 * k + 1] : inv[2 * k + 1]);
  }
}

void orc_sincos2pif(float u, float* c_out, float* s_out) {
  float cosc[ORC_TRIG_TERMS], sinc[ORC_TRIG_TERMS];
  orc_trig_coefs(cosc, sinc);
  float x = u * 4.0f;
  int q = (int)x;
  float f = x - (float)q;
  float th = f * ORC_PI_2F;
  float z = th * th;
  float cs = cosc[ORC_TRIG_TERMS - 1];
  float sn = sinc[ORC_TRIG_TERMS - 1];
  for (int k = ORC_TRIG_TERMS - 2; k >= 0; --k) {
    cs = fmaf(cs, z, cosc[k]);
    sn = fmaf(sn, z, sinc[k]);
  }
  sn = sn * th;
  switch (q & 3) {
    case 0: *c_out = cs; *s_out = sn; break;
    case 1: *c_out = -sn; *s_out = cs; break;
    case 2: *c_out = -cs; *s_out = -sn; break;
    default: *c_out = sn; *s_out = -cs; break;
  }
}

/* ------------------------------------------------------------------------- */
/* Random direction for (tree t, node key, try j): the direction draw of    */
/* Algorithms 1 and 2 (Sec. 2), all in FP32: g_{2i}, g_{2i+1} by             */
/* Box-Muller from the top 24 bits of words c = 2i and c = 2i+1; then         */
/* s = sequential fmaf sum of g_k^2, inv = 1 / sqrtf(s), r_k = g_k * inv.     */
/* r is returned as doubles (exactly the FP32 values).                        */
/* ------------------------------------------------------------------------- */
void orc_direction(uint64_t seed, uint64_t t, uint64_t key, uint64_t j, int d,
                   double* r) {
  float* g = (float*)malloc(sizeof(float) * (size_t)(d + 1));
  for (int i = 0; 2 * i < d; ++i) {
    uint64_t w1 = orc_word(seed, ORC_TAG_DIR, t, key, j, (uint64_t)(2 * i));
    uint64_t w2 = orc_word(seed, ORC_TAG_DIR, t, key, j, (uint64_t)(2 * i + 1));
    float u1 = (float)((w1 >> 40) + 1) * 0x1p-24f; /* (0, 1] */
    float u2 = (float)(w2 >> 40) * 0x1p-24f;       /* [0, 1) */
    float rho = sqrtf(-2.0f * orc_lnf(u1));
    float c, s;
    orc_sincos2pif(u2, &c, &s);
    g[2 * i] = rho * c;
    if (2 * i + 1 < d) g[2 * i + 1] = rho * s;
  }
  float ss = 0.0f;
  for (int k = 0; k < d; ++k) ss = fmaf(g[k], g[k], ss);
  if (ss == 0.0f) { /* unreachable in practice: every Gaussian pair zero */
    for (int k = 0; k < d; ++k) r[k] = 0.0;
    r[0] = 1.0;
    free(g);
    return;
  }
  float inv = 1.0f / sqrtf(ss);
  for (int k = 0; k < d; ++k) r[k] = (double)(g[k] * inv);
  free(g);
}

/* Projection of x on the direction r (Sec. 2, Algorithms 1-2). */
double orc_proj(const float* x, const double* r, int d) {
  double p = 0.0;
  for (int k = 0; k < d; ++k) p = fma((double)x[k], r[k], p);
  return p;
}

/* ------------------------------------------------------------------------- */
/* Canonical-order FP64 sum.  Chunks of 4096 positions; inside a chunk lane  */
/* l (0..31) sums positions l, l+32, ... sequentially from +0.0; the 32 lane  */
/* sums are folded pairwise s_l += s_{l+16}, then +8, +4, +2, +1.  More than  */
/* one chunk: the chunk sums are reduced by the same rule, recursively.       */
/* ------------------------------------------------------------------------- */
static double orc_chunk_sum(const double* v, int64_t len) {
  double s[32];
  for (int l = 0; l < 32; ++l) {
    double a = 0.0;
    for (int64_t k = l; k < len; k += 32) a = a + v[k];
    s[l] = a;
  }
  for (int off = 16; off >= 1; off >>= 1)
    for (int l = 0; l < off; ++l) s[l] = s[l] + s[l + off];
  return s[0];
}

double orc_csum(const double* v, int64_t m) {
  if (m <= ORC_CHUNK) return orc_chunk_sum(v, m);
  int64_t nc = (m + ORC_CHUNK - 1) / ORC_CHUNK;
  double* part = (double*)malloc(sizeof(double) * (size_t)nc);
  for (int64_t c = 0; c < nc; ++c) {
    int64_t len = m - c * ORC_CHUNK;
    if (len > ORC_CHUNK) len = ORC_CHUNK;
    part[c] = orc_chunk_sum(v + c * ORC_CHUNK, len);
  }
  double r = orc_csum(part, nc);
  free(part);
  return r;
}

/* Canonical squared distance d32 between two FP32 rows. */
float orc_d32(const float* x, const float* y, int d) {
  float s = 0.0f;
  for (int k = 0; k < d; ++k) {
    float e = x[k] - y[k];
    s = fmaf(e, e, s);
  }
  return s;
}

/* ------------------------------------------------------------------------- */
/* Forest.                                                                   */
/* ------------------------------------------------------------------------- */
typedef struct {
  uint64_t key;
  int64_t begin, len; /* segment of the tree's perm */
  int32_t depth;
  int32_t leaf;       /* 1: leaf (len <= L) */
  int32_t jstar;      /* chosen try, -1 if none had V > 0 */
  int32_t flag;       /* 1: rank split (degenerate node) */
  int32_t attempt;    /* accepted split attempt, -1 for rank split */
  int32_t pad;
  double c;           /* split point (NaN for rank split) */
  double a, b;        /* min / max of the chosen projections */
  int64_t left, right;
  int64_t dir;        /* offset of r* in the tree's direction store, -1 */
} orc_node;

typedef struct {
  orc_node* nodes;
  int64_t n_nodes, cap_nodes;
  double* dirs;
  int64_t n_dirs, cap_dirs; /* counted in directions of length d */
  int32_t* perm;            /* n */
} orc_tree;

typedef struct {
  int64_t n;
  int32_t d, T, L, ntry;
  int32_t t0;         /* global index of the first tree (draws are keyed by it) */
  int32_t split_rule; /* 0: c ~ U[a, b]; 1: median of the projections */
  uint64_t seed;
  orc_tree* trees;
  const float* X; /* borrowed: valid only during orc_build */
} orc_forest;

static int64_t orc_push_node(orc_tree* tr, orc_node nd) {
  if (tr->n_nodes == tr->cap_nodes) {
    tr->cap_nodes = tr->cap_nodes ? 2 * tr->cap_nodes : 64;
    tr->nodes = (orc_node*)realloc(tr->nodes, sizeof(orc_node) * (size_t)tr->cap_nodes);
  }
  tr->nodes[tr->n_nodes] = nd;
  return tr->n_nodes++;
}

static int64_t orc_push_dir(orc_tree* tr, const double* r, int d) {
  if (tr->n_dirs == tr->cap_dirs) {
    tr->cap_dirs = tr->cap_dirs ? 2 * tr->cap_dirs : 64;
    tr->dirs = (double*)realloc(tr->dirs, sizeof(double) * (size_t)d * (size_t)tr->cap_dirs);
  }
  memcpy(tr->dirs + (size_t)d * (size_t)tr->n_dirs, r, sizeof(double) * (size_t)d);
  return tr->n_dirs++;
}

/* (p[i], id[i]) < (p[j], id[j]) in the order the median rule uses: by
   projection, ties by the point's index. */
static int orc_key_less(const double* p, const int32_t* id, int64_t i, int64_t j) {
  return p[i] < p[j] || (p[i] == p[j] && id[i] < id[j]);
}

/* ord[0..m) = 0..m-1 sorted by (p, id): plain bottom-up merge sort. */
static void orc_sort_by_key(const double* p, const int32_t* id, int64_t m, int64_t* ord) {
  int64_t* buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  for (int64_t i = 0; i < m; ++i) ord[i] = i;
  for (int64_t w = 1; w < m; w *= 2) {
    for (int64_t lo = 0; lo < m; lo += 2 * w) {
      int64_t mid = lo + w < m ? lo + w : m, hi = lo + 2 * w < m ? lo + 2 * w : m;
      int64_t a = lo, b = mid, k = lo;
      while (a < mid && b < hi) buf[k++] = orc_key_less(p, id, ord[b], ord[a]) ? ord[b++] : ord[a++];
      while (a < mid) buf[k++] = ord[a++];
      while (b < hi) buf[k++] = ord[b++];
    }
    memcpy(ord, buf, sizeof(int64_t) * (size_t)m);
  }
  free(buf);
}

/* Split one node (Algorithm 1 body with Algorithm 2 for the direction). */
static void orc_split(const orc_forest* F, orc_tree* tr, int64_t t, int64_t ni,
                      double* pbuf, double* qbuf, double* rbuf, int32_t* tmp) {
  const int d = F->d, ntry = F->ntry;
  orc_node* nd = &tr->nodes[ni];
  const int64_t m = nd->len, b0 = nd->begin;
  int32_t* mem = tr->perm + b0;

  /* Algorithm 2: nTry directions, keep the first with the largest dispersion. */
  double best = 0.0;
  int jstar = -1;
  for (int j = 0; j < ntry; ++j) {
    double* r = rbuf + (size_t)j * d;
    double* p = pbuf + (size_t)j * m;
    orc_direction(F->seed, (uint64_t)(t + F->t0), nd->key, (uint64_t)j, d, r);
    for (int64_t i = 0; i < m; ++i) p[i] = orc_proj(F->X + (size_t)mem[i] * d, r, d);
    double S = orc_csum(p, m);
    double mu = S / (double)m;
    for (int64_t i = 0; i < m; ++i) {
      double e = p[i] - mu;
      qbuf[i] = e * e;
    }
    double V = orc_csum(qbuf, m);
    if (V > best) {
      best = V;
      jstar = j;
    }
  }
  nd->jstar = jstar;

  /* Algorithm 1: a = min, b = max of the projections, c ~ U[a, b]. */
  int accepted = 0;
  double c = NAN, a = NAN, b = NAN;
  const double* p = NULL;
  if (jstar >= 0) {
    p = pbuf + (size_t)jstar * m;
    a = p[0];
    b = p[0];
    for (int64_t i = 1; i < m; ++i) {
      if (p[i] < a) a = p[i];
      if (p[i] > b) b = p[i];
    }
    for (int att = 0; F->split_rule == 0 && att < ORC_SPLIT_ATTEMPTS; ++att) {
      double u = orc_u53(orc_word(F->seed, ORC_TAG_SPLIT, (uint64_t)(t + F->t0), nd->key,
                                  (uint64_t)att, 0));
      double cc = fma(u, b - a, a);
      if (cc > a && cc <= b) {
        c = cc;
        nd->attempt = att;
        accepted = 1;
        break;
      }
    }
  }
  nd->a = a;
  nd->b = b;

  /* Median rule (Sec. 2, the other usual split point): the floor(m/2) points
     smallest in (projection, index) order go left, node order kept on each
     side; c is the projection of the first point that goes right, so a
     query goes left iff its projection is below the median. */
  int64_t nl = 0;
  if (F->split_rule == 1 && jstar >= 0) {
    int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    uint8_t* left = (uint8_t*)calloc((size_t)m, 1);
    orc_sort_by_key(p, mem, m, ord);
    const int64_t h = m / 2;
    for (int64_t k = 0; k < h; ++k) left[ord[k]] = 1;
    c = p[ord[h]];
    int64_t w = 0;
    for (int64_t i = 0; i < m; ++i)
      if (left[i]) tmp[w++] = mem[i];
    nl = w;
    for (int64_t i = 0; i < m; ++i)
      if (!left[i]) tmp[w++] = mem[i];
    free(ord);
    free(left);
    nd->c = c;
    nd->flag = 0;
    nd->attempt = -1;
    nd->dir = orc_push_dir(tr, rbuf + (size_t)jstar * d, d);
    nd = &tr->nodes[ni];
  } else if (accepted) {
    int64_t w = 0;
    for (int64_t i = 0; i < m; ++i)
      if (p[i] < c) tmp[w++] = mem[i];
    nl = w;
    for (int64_t i = 0; i < m; ++i)
      if (!(p[i] < c)) tmp[w++] = mem[i];
    nd->c = c;
    nd->flag = 0;
    nd->dir = orc_push_dir(tr, rbuf + (size_t)jstar * d, d);
    nd = &tr->nodes[ni];
  } else { /* degenerate node: first floor(m/2) positions go left */
    nl = m / 2;
    for (int64_t i = 0; i < m; ++i) tmp[i] = mem[i];
    nd->c = NAN;
    nd->flag = 1;
    nd->attempt = -1;
    nd->dir = -1;
  }
  memcpy(mem, tmp, sizeof(int32_t) * (size_t)m);

  orc_node L = {0}, R = {0};
  L.key = orc_child_key(nd->key, 0);
  R.key = orc_child_key(nd->key, 1);
  L.begin = b0;
  L.len = nl;
  R.begin = b0 + nl;
  R.len = m - nl;
  L.depth = R.depth = nd->depth + 1;
  L.jstar = R.jstar = -1;
  L.attempt = R.attempt = -1;
  L.left = L.right = R.left = R.right = -1;
  L.dir = R.dir = -1;
  L.c = R.c = L.a = L.b = R.a = R.b = NAN;
  int64_t li = orc_push_node(tr, L);
  int64_t ri = orc_push_node(tr, R);
  tr->nodes[ni].left = li;
  tr->nodes[ni].right = ri;
}

static void orc_grow_tree(const orc_forest* F, int64_t t) {
  orc_tree* tr = &F->trees[t];
  const int64_t n = F->n;
  tr->perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) tr->perm[i] = (int32_t)i;
  orc_node root = {0};
  root.key = 1;
  root.begin = 0;
  root.len = n;
  root.jstar = -1;
  root.attempt = -1;
  root.left = root.right = -1;
  root.dir = -1;
  root.c = root.a = root.b = NAN;
  orc_push_node(tr, root);

  double* pbuf = (double*)malloc(sizeof(double) * (size_t)n * (size_t)F->ntry);
  double* qbuf = (double*)malloc(sizeof(double) * (size_t)n);
  double* rbuf = (double*)malloc(sizeof(double) * (size_t)F->d * (size_t)F->ntry);
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);

  /* Working set W of Algorithm 1, kept as a stack (the pick order does not
     matter because every draw is keyed by the node). */
  int64_t cap = 64, top = 0;
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
  stack[top++] = 0;
  while (top > 0) {
    int64_t ni = stack[--top];
    if (tr->nodes[ni].len <= F->L) {
      tr->nodes[ni].leaf = 1;
      continue;
    }
    orc_split(F, tr, t, ni, pbuf, qbuf, rbuf, tmp);
    if (top + 2 > cap) {
      cap *= 2;
      stack = (int64_t*)realloc(stack, sizeof(int64_t) * (size_t)cap);
    }
    stack[top++] = tr->nodes[ni].right;
    stack[top++] = tr->nodes[ni].left;
  }
  free(stack);
  free(pbuf);
  free(qbuf);
  free(rbuf);
  free(tmp);
}

/* Build trees t0 .. t0 + T - 1 of the ensemble (Algorithm 3, first loop):
   every draw of tree t is keyed by its global index t, so these are exactly
   the trees a forest of t0 + T trees holds at those indexes.  Trees are
   independent, so with OpenMP they are grown one per thread -- the multicore
   scheme of Sec. 5.3. */
orc_forest* orc_build_range(const float* X, int64_t n, int32_t d, int32_t t0, int32_t T,
                            int32_t L, int32_t ntry, uint64_t seed, int32_t threads,
                            int32_t split_rule) {
  if (!X || n < 1 || d < 1 || t0 < 0 || T < 1 || L < 1 || ntry < 1) return NULL;
  if (split_rule < 0 || split_rule > 1) return NULL;
  orc_forest* F = (orc_forest*)calloc(1, sizeof(orc_forest));
  F->t0 = t0;
  F->split_rule = split_rule;
  F->n = n;
  F->d = d;
  F->T = T;
  F->L = L;
  F->ntry = ntry;
  F->seed = seed;
  F->X = X;
  F->trees = (orc_tree*)calloc((size_t)T, sizeof(orc_tree));
#ifdef _OPENMP
  if (threads < 1) threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
#endif
  for (int64_t t = 0; t < T; ++t) orc_grow_tree(F, t);
  (void)threads;
  F->X = NULL;
  return F;
}

/* The first T trees of the ensemble. */
orc_forest* orc_build(const float* X, int64_t n, int32_t d, int32_t T, int32_t L,
                      int32_t ntry, uint64_t seed, int32_t threads, int32_t split_rule) {
  return orc_build_range(X, n, d, 0, T, L, ntry, seed, threads, split_rule);
}

void orc_free(orc_forest* F) {
  if (!F) return;
  for (int32_t t = 0; t < F->T; ++t) {
    free(F->trees[t].nodes);
    free(F->trees[t].dirs);
    free(F->trees[t].perm);
  }
  free(F->trees);
  free(F);
}

int64_t orc_n_nodes(const orc_forest* F, int32_t t) { return F->trees[t].nodes ? F->trees[t].n_nodes : 0; }

void orc_get_perm(const orc_forest* F, int32_t t, int32_t* out) {
  memcpy(out, F->trees[t].perm, sizeof(int32_t) * (size_t)F->n);
}

/* Node table of tree t: int64 fields [key, begin, len, depth, leaf, jstar,
   flag, attempt, left, right] per node into I (10 per node) and double fields
   [c, a, b] into Dv (3 per node). */
void orc_get_nodes(const orc_forest* F, int32_t t, int64_t* I, double* Dv) {
  const orc_tree* tr = &F->trees[t];
  for (int64_t i = 0; i < tr->n_nodes; ++i) {
    const orc_node* nd = &tr->nodes[i];
    int64_t* o = I + 10 * i;
    o[0] = (int64_t)nd->key;
    o[1] = nd->begin;
    o[2] = nd->len;
    o[3] = nd->depth;
    o[4] = nd->leaf;
    o[5] = nd->jstar;
    o[6] = nd->flag;
    o[7] = nd->attempt;
    o[8] = nd->left;
    o[9] = nd->right;
    Dv[3 * i + 0] = nd->c;
    Dv[3 * i + 1] = nd->a;
    Dv[3 * i + 2] = nd->b;
  }
}

/* Chosen direction r* of node i of tree t (zeros for leaves / rank splits). */
void orc_get_node_dir(const orc_forest* F, int32_t t, int64_t i, double* r) {
  const orc_tree* tr = &F->trees[t];
  const orc_node* nd = &tr->nodes[i];
  if (nd->dir < 0) {
    for (int k = 0; k < F->d; ++k) r[k] = 0.0;
    return;
  }
  memcpy(r, tr->dirs + (size_t)F->d * (size_t)nd->dir, sizeof(double) * (size_t)F->d);
}

/* ------------------------------------------------------------------------- */
/* K nearest by (d32, idx) ascending: insertion into a sorted list of K.      */
/* ------------------------------------------------------------------------- */
static void orc_topk_insert(float* kd, int32_t* ki, int K, float dv, int32_t j) {
  if (!(dv < kd[K - 1] || (dv == kd[K - 1] && (ki[K - 1] < 0 || j < ki[K - 1])))) return;
  int p = K - 1;
  while (p > 0 && (dv < kd[p - 1] || (dv == kd[p - 1] && (ki[p - 1] < 0 || j < ki[p - 1])))) {
    kd[p] = kd[p - 1];
    ki[p] = ki[p - 1];
    --p;
  }
  kd[p] = dv;
  ki[p] = j;
}

/* Candidate set of one query: the union over trees of its leaves
   (Algorithm 3: N_q = U_i N^i), then the K closest.  self < 0: nothing is
   excluded (a query that is not a data point). */
static void orc_knn_from_union(const float* X, int d, const float* q, int32_t self,
                               int32_t* const* leaf_members, const int64_t* leaf_len,
                               int32_t T, int32_t K, int32_t* stamp, int32_t stamp_id,
                               int32_t* idx_out, float* dist_out, int squared) {
  float* kd = (float*)malloc(sizeof(float) * (size_t)K);
  for (int k = 0; k < K; ++k) {
    kd[k] = INFINITY;
    idx_out[k] = -1;
  }
  for (int32_t t = 0; t < T; ++t) {
    const int32_t* mem = leaf_members[t];
    for (int64_t a = 0; a < leaf_len[t]; ++a) {
      int32_t j = mem[a];
      if (j == self || stamp[j] == stamp_id) continue;
      stamp[j] = stamp_id;
      orc_topk_insert(kd, idx_out, K, orc_d32(q, X + (size_t)j * d, d), j);
    }
  }
  for (int k = 0; k < K; ++k)
    dist_out[k] = idx_out[k] < 0 ? INFINITY : (squared ? kd[k] : sqrtf(kd[k]));
  free(kd);
}

/* All-kNN, Q = U (Algorithm 3).  Each point i is excluded from its own list;
   lists shorter than K are padded with (-1, +inf).  X must be the data the
   forest was built on. */
void orc_all_knn(const orc_forest* F, const float* X, int32_t K, int32_t* idx,
                 float* dist, int32_t threads) {
  const int64_t n = F->n;
  const int T = F->T;
  /* leaf segment of each point in each tree */
  int64_t* lb = (int64_t*)malloc(sizeof(int64_t) * (size_t)n * (size_t)T);
  int64_t* ll = (int64_t*)malloc(sizeof(int64_t) * (size_t)n * (size_t)T);
  for (int t = 0; t < T; ++t) {
    const orc_tree* tr = &F->trees[t];
    for (int64_t i = 0; i < tr->n_nodes; ++i) {
      const orc_node* nd = &tr->nodes[i];
      if (!nd->leaf) continue;
      for (int64_t a = 0; a < nd->len; ++a) {
        int32_t j = tr->perm[nd->begin + a];
        lb[(size_t)j * T + t] = nd->begin;
        ll[(size_t)j * T + t] = nd->len;
      }
    }
  }
#ifdef _OPENMP
  if (threads < 1) threads = 1;
#pragma omp parallel num_threads(threads)
#endif
  {
    int32_t* stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) stamp[i] = -1;
    int32_t** mem = (int32_t**)malloc(sizeof(int32_t*) * (size_t)T);
    int64_t* len = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
    for (int64_t i = 0; i < n; ++i) {
      for (int t = 0; t < T; ++t) {
        mem[t] = F->trees[t].perm + lb[(size_t)i * T + t];
        len[t] = ll[(size_t)i * T + t];
      }
      orc_knn_from_union(X, F->d, X + (size_t)i * F->d, (int32_t)i, mem, len, T, K, stamp,
                         (int32_t)i, idx + (size_t)i * K, dist + (size_t)i * K, 0);
    }
    free(stamp);
    free(mem);
    free(len);
  }
  (void)threads;
}

/* All-kNN answers for the data points rows[0..nr) only (same definition as
   orc_all_knn; used to check large instances on a sample).  squared = 1
   reports the d32 key itself instead of its square root. */
static void orc_all_knn_rows_impl(const orc_forest* F, const float* X, const int32_t* rows,
                                  int64_t nr, int32_t K, int32_t* idx, float* dist,
                                  int32_t threads, int squared) {
  const int64_t n = F->n;
  const int T = F->T;
  /* position of every point in every tree's permutation */
  int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * (size_t)T);
  int64_t** leaf_b = (int64_t**)malloc(sizeof(int64_t*) * (size_t)T);
  int64_t** leaf_l = (int64_t**)malloc(sizeof(int64_t*) * (size_t)T);
  for (int t = 0; t < T; ++t) {
    const orc_tree* tr = &F->trees[t];
    for (int64_t a = 0; a < n; ++a) pos[(size_t)tr->perm[a] * T + t] = (int32_t)a;
    leaf_b[t] = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    leaf_l[t] = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < tr->n_nodes; ++i) {
      const orc_node* nd = &tr->nodes[i];
      if (!nd->leaf) continue;
      for (int64_t a = 0; a < nd->len; ++a) {
        leaf_b[t][nd->begin + a] = nd->begin;
        leaf_l[t][nd->begin + a] = nd->len;
      }
    }
  }
#ifdef _OPENMP
  if (threads < 1) threads = 1;
#pragma omp parallel num_threads(threads)
#endif
  {
    int32_t* stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) stamp[i] = -1;
    int32_t** mem = (int32_t**)malloc(sizeof(int32_t*) * (size_t)T);
    int64_t* len = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8)
#endif
    for (int64_t r = 0; r < nr; ++r) {
      const int32_t i = rows[r];
      for (int t = 0; t < T; ++t) {
        const int64_t a = pos[(size_t)i * T + t];
        mem[t] = F->trees[t].perm + leaf_b[t][a];
        len[t] = leaf_l[t][a];
      }
      orc_knn_from_union(X, F->d, X + (size_t)i * F->d, i, mem, len, T, K, stamp, (int32_t)r,
                         idx + (size_t)r * K, dist + (size_t)r * K, squared);
    }
    free(stamp);
    free(mem);
    free(len);
  }
  for (int t = 0; t < T; ++t) {
    free(leaf_b[t]);
    free(leaf_l[t]);
  }
  free(leaf_b);
  free(leaf_l);
  free(pos);
  (void)threads;
}

void orc_all_knn_rows(const orc_forest* F, const float* X, const int32_t* rows, int64_t nr,
                      int32_t K, int32_t* idx, float* dist, int32_t threads) {
  orc_all_knn_rows_impl(F, X, rows, nr, K, idx, dist, threads, 0);
}

/* The same lists as orc_all_knn_rows with the squared key d32 in place of the
   distance: the per-point lists a set of trees contributes to a union over
   more trees (a forest split into groups of trees). */
void orc_all_knn_keys(const orc_forest* F, const float* X, const int32_t* rows, int64_t nr,
                      int32_t K, int32_t* idx, float* d32, int32_t threads) {
  orc_all_knn_rows_impl(F, X, rows, nr, K, idx, d32, threads, 1);
}

/* Drop a point through tree t (Algorithm 3, "let q fall through tree t_i"):
   at an internal node go left iff r* . q < c; a rank-split node sends every
   query left.  Returns the leaf's node index. */
int64_t orc_route(const orc_forest* F, int32_t t, const float* q) {
  const orc_tree* tr = &F->trees[t];
  int64_t i = 0;
  while (!tr->nodes[i].leaf) {
    const orc_node* nd = &tr->nodes[i];
    if (nd->flag) {
      i = nd->left;
      continue;
    }
    double p = orc_proj(q, tr->dirs + (size_t)F->d * (size_t)nd->dir, F->d);
    i = (p < nd->c) ? nd->left : nd->right;
  }
  return i;
}

/* kNN of m new points Q in the data X (Algorithm 3 with Q outside U). */
void orc_query(const orc_forest* F, const float* X, const float* Q, int64_t m,
               int32_t K, int32_t* idx, float* dist, int32_t threads) {
  const int T = F->T;
#ifdef _OPENMP
  if (threads < 1) threads = 1;
#pragma omp parallel num_threads(threads)
#endif
  {
    int32_t* stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)F->n);
    for (int64_t i = 0; i < F->n; ++i) stamp[i] = -1;
    int32_t** mem = (int32_t**)malloc(sizeof(int32_t*) * (size_t)T);
    int64_t* len = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
    for (int64_t qi = 0; qi < m; ++qi) {
      const float* q = Q + (size_t)qi * F->d;
      for (int t = 0; t < T; ++t) {
        const orc_tree* tr = &F->trees[t];
        const orc_node* lf = &tr->nodes[orc_route(F, t, q)];
        mem[t] = tr->perm + lf->begin;
        len[t] = lf->len;
      }
      orc_knn_from_union(X, F->d, q, -1, mem, len, T, K, stamp, (int32_t)qi,
                         idx + (size_t)qi * K, dist + (size_t)qi * K, 0);
    }
    free(stamp);
    free(mem);
    free(len);
  }
  (void)threads;
}

/* Exact brute-force kNN under the (d32, idx) order for the rows `rows` (nr of
   them) against all n points; exclude_self drops j == row.  Also reports the
   FP64 Euclidean distance of every returned neighbour in dist64. */
void orc_brute_knn(const float* X, int64_t n, int32_t d, const float* Q, int64_t nr,
                   const int32_t* self_idx, int32_t K, int32_t* idx, float* dist,
                   double* dist64, int32_t threads) {
#ifdef _OPENMP
  if (threads < 1) threads = 1;
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads)
#endif
  for (int64_t r = 0; r < nr; ++r) {
    const float* q = Q + (size_t)r * d;
    int32_t self = self_idx ? self_idx[r] : -1;
    float* kd = (float*)malloc(sizeof(float) * (size_t)K);
    int32_t* ki = idx + (size_t)r * K;
    for (int k = 0; k < K; ++k) {
      kd[k] = INFINITY;
      ki[k] = -1;
    }
    for (int64_t j = 0; j < n; ++j) {
      if ((int32_t)j == self) continue;
      orc_topk_insert(kd, ki, K, orc_d32(q, X + (size_t)j * d, d), (int32_t)j);
    }
    for (int k = 0; k < K; ++k) {
      if (ki[k] < 0) {
        dist[(size_t)r * K + k] = INFINITY;
        dist64[(size_t)r * K + k] = INFINITY;
        continue;
      }
      dist[(size_t)r * K + k] = sqrtf(kd[k]);
      const float* y = X + (size_t)ki[k] * d;
      double s = 0.0;
      for (int c = 0; c < d; ++c) {
        double e = (double)q[c] - (double)y[c];
        s = fma(e, e, s);
      }
      dist64[(size_t)r * K + k] = sqrt(s);
    }
    free(kd);
  }
  (void)threads;
}

int orc_have_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}
