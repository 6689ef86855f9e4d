/*
 * Seam-carving oracle: plain, slow, single-threaded C.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load this file;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg do. It shares no code,
 * header, table or helper with the CUDA library, and it never reads values produced by it.
 *
 * It states, in the order and notation of the paper (arXiv 2410.21207, "Analysis of Different
 * Algorithmic Design Techniques for Seam Carving"), what the hot path computes:
 *   - energy e1: sum of the magnitudes of the x and y partial derivatives ("Energy Mapping");
 *   - Algorithm 1 (brute force), Algorithm 2 (greedy), Algorithm 3 (dynamic programming) for
 *     one minimum vertical seam ("Design Techniques");
 *   - removal: every pixel of a row right of the seam moves one column left ("Removal of Seams");
 *   - the repeated loop, with horizontal seams found on the transposed image ("Design
 *     Techniques", opening paragraph: rows and columns swap).
 *
 * Where the paper is silent or garbled, the readings are:
 *   R1 energy: per channel |I(i,j+1)-I(i,j-1)| + |I(i+1,j)-I(i-1,j)|, summed over the C channels,
 *      integer, no scaling; indices outside the image are clamped to the border (edge
 *      replication), so a 1-wide image has a zero x term.
 *   R2 DP first row: M(0,j) = e(0,j) (Algorithm 3 starts at the second row and leaves the first
 *      uninitialised).
 *   R3 neighbours outside [0,W) are excluded (never wrapped).
 *   R4 ties: the leftmost of (j-1, j, j+1) wins, and the leftmost minimum of the last row wins.
 *   R5 backtrack: seam[H-1] = argmin of the last row, then seam[i-1] = B(i, seam[i]) (the printed
 *      loop is off by one).
 *   R6 brute force: every 8-connected path, bottom column ascending, each step up choosing
 *      col-1, col, col+1 ascending (in range only), adding the energy of every row; a path
 *      replaces the best only when strictly cheaper.
 *   R7 greedy: starts at the leftmost minimum of the bottom row, climbs by the leftmost minimum
 *      of the in-range upper neighbours; its cost is the sum of e along its path.
 *   R8 horizontal seams: transpose, remove vertical seams, transpose back; all vertical seams
 *      are removed before the horizontal ones.
 *   R9 seam insertion (enlargement, which the paper names as a use of seams without giving its
 *      steps): to widen by k (1 <= k <= W-1), take the first k seams that the loop would remove
 *      from the W-wide image, each mapped back to the input column it deletes; after every input
 *      pixel on one of them insert one pixel whose channels are the rounded-up mean
 *      (a + b + 1) / 2 of that pixel and its right neighbour (the pixel itself at the last
 *      column, by the border clamp of R1).
 *   R10 forward energy (the paper cites it as an alternative criterion without a formula): the
 *      cost of a seam is the sum, over the pixel pairs that become adjacent when it is removed, of
 *      their L1 colour difference. Per pixel (i, j) with the seam arriving from (i-1, j') this is
 *      CU = |I(i,j+1) - I(i,j-1)| (0 when j is the first or last column: no new horizontal pair),
 *      plus DL = |I(i-1,j) - I(i,j-1)| when j' = j-1, or DR = |I(i-1,j) - I(i,j+1)| when j' = j+1;
 *      row 0 costs CU only. The DP is Algorithm 3 with these per-direction costs, with R3-R5.
 * Energies and costs are exact integers (int64 here), so no rounding question arises.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- energy e1 (Energy Mapping, list item e1; reading R1) ---- */
static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }
static int absi(int x) { return x < 0 ? -x : x; }

void orc_energy(const uint8_t *img, int H, int W, int C, uint16_t *e) {
  for (int i = 0; i < H; ++i) {
    int iu = clampi(i - 1, 0, H - 1), id = clampi(i + 1, 0, H - 1);
    for (int j = 0; j < W; ++j) {
      int jl = clampi(j - 1, 0, W - 1), jr = clampi(j + 1, 0, W - 1);
      int s = 0;
      for (int c = 0; c < C; ++c) {
        int dx = (int)img[((size_t)i * W + jr) * C + c] - (int)img[((size_t)i * W + jl) * C + c];
        int dy = (int)img[((size_t)id * W + j) * C + c] - (int)img[((size_t)iu * W + j) * C + c];
        s += absi(dx) + absi(dy);
      }
      e[(size_t)i * W + j] = (uint16_t)s;
    }
  }
}

/* ---- Algorithm 3: dynamic programming (DP Seam Carving; recurrence
 *      M(i,j) = e(i,j) + min(M(i-1,j-1), M(i-1,j), M(i-1,j+1)); readings R2-R5) ----
 * M and B are full H x W tables, as in the algorithm. Returns the seam's total cost. */
int64_t orc_dp_seam(const uint16_t *e, int H, int W, int32_t *seam) {
  int64_t *M = (int64_t *)malloc(sizeof(int64_t) * (size_t)H * W);
  int32_t *B = (int32_t *)malloc(sizeof(int32_t) * (size_t)H * W);
  for (int j = 0; j < W; ++j) { M[j] = e[j]; B[j] = -1; }
  for (int i = 1; i < H; ++i) {
    for (int j = 0; j < W; ++j) {
      int best = -1;
      int64_t bestv = 0;
      for (int jp = j - 1; jp <= j + 1; ++jp) {          /* candidates in the order j-1, j, j+1 */
        if (jp < 0 || jp >= W) continue;                 /* R3 */
        int64_t v = M[(size_t)(i - 1) * W + jp];
        if (best < 0 || v < bestv) { best = jp; bestv = v; }   /* strict: the leftmost wins (R4) */
      }
      B[(size_t)i * W + j] = best;
      M[(size_t)i * W + j] = (int64_t)e[(size_t)i * W + j] + bestv;
    }
  }
  int jstar = 0;
  for (int j = 1; j < W; ++j)
    if (M[(size_t)(H - 1) * W + j] < M[(size_t)(H - 1) * W + jstar]) jstar = j;
  int64_t cost = M[(size_t)(H - 1) * W + jstar];
  seam[H - 1] = jstar;
  for (int i = H - 1; i >= 1; --i) seam[i - 1] = B[(size_t)i * W + seam[i]];   /* R5 */
  free(M);
  free(B);
  return cost;
}

/* The last row of M (the cumulative cost table of Algorithm 3), for tests of the cost table. */
void orc_dp_last_row(const uint16_t *e, int H, int W, int64_t *last) {
  int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * W);
  int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * W);
  for (int j = 0; j < W; ++j) prev[j] = e[j];
  for (int i = 1; i < H; ++i) {
    for (int j = 0; j < W; ++j) {
      int64_t b = prev[j];
      if (j > 0 && prev[j - 1] < b) b = prev[j - 1];
      if (j + 1 < W && prev[j + 1] < b) b = prev[j + 1];
      cur[j] = (int64_t)e[(size_t)i * W + j] + b;
    }
    int64_t *t = prev; prev = cur; cur = t;
  }
  memcpy(last, prev, sizeof(int64_t) * W);
  free(prev);
  free(cur);
}

/* ---- Algorithm 2: greedy (Greedy Seam Carving; readings R4, R7) ---- */
int64_t orc_greedy_seam(const uint16_t *e, int H, int W, int32_t *seam) {
  int start = 0;
  for (int j = 1; j < W; ++j)
    if (e[(size_t)(H - 1) * W + j] < e[(size_t)(H - 1) * W + start]) start = j;
  int64_t cost = e[(size_t)(H - 1) * W + start];
  seam[H - 1] = start;
  for (int i = H - 2; i >= 0; --i) {
    int best = -1;
    for (int jp = start - 1; jp <= start + 1; ++jp) {
      if (jp < 0 || jp >= W) continue;
      if (best < 0 || e[(size_t)i * W + jp] < e[(size_t)i * W + best]) best = jp;
    }
    start = best;
    seam[i] = start;
    cost += e[(size_t)i * W + start];
  }
  return cost;
}

/* ---- Algorithm 1: brute force (BruteForce Seam Carving; reading R6) ---- */
typedef struct {
  const uint16_t *e;
  int H, W;
  int64_t best;
  int have;
  int32_t *path;     /* current path, indexed by row */
  int32_t *bestpath;
  int64_t leaves;    /* number of complete paths visited */
} brute_ctx;

static void brute_helper(brute_ctx *b, int row, int col, int64_t cost) {
  cost += b->e[(size_t)row * b->W + col];
  b->path[row] = col;
  if (row == 0) {
    b->leaves++;
    if (!b->have || cost < b->best) {
      b->have = 1;
      b->best = cost;
      memcpy(b->bestpath, b->path, sizeof(int32_t) * b->H);
    }
    return;
  }
  for (int nb = col - 1; nb <= col + 1; ++nb) {
    if (nb < 0 || nb >= b->W) continue;
    brute_helper(b, row - 1, nb, cost);
  }
}

/* Returns the minimum cost; *leaves_out (nullable) receives the number of paths enumerated. */
int64_t orc_brute_seam(const uint16_t *e, int H, int W, int32_t *seam, int64_t *leaves_out) {
  brute_ctx b;
  b.e = e; b.H = H; b.W = W; b.best = 0; b.have = 0; b.leaves = 0;
  b.path = (int32_t *)malloc(sizeof(int32_t) * H);
  b.bestpath = seam;
  for (int col = 0; col < W; ++col) brute_helper(&b, H - 1, col, 0);
  if (leaves_out) *leaves_out = b.leaves;
  free(b.path);
  return b.best;
}

/* ---- Removal of Seams: each row loses the pixel at seam[i]; the rest keep their order ---- */
void orc_remove_seam(const uint8_t *img, int H, int W, int C, const int32_t *seam, uint8_t *out) {
  for (int i = 0; i < H; ++i) {
    int o = 0;
    for (int j = 0; j < W; ++j) {
      if (j == seam[i]) continue;
      for (int c = 0; c < C; ++c) out[((size_t)i * (W - 1) + o) * C + c] = img[((size_t)i * W + j) * C + c];
      ++o;
    }
  }
}

void orc_transpose(const uint8_t *img, int H, int W, int C, uint8_t *out) {
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j)
      for (int c = 0; c < C; ++c) out[((size_t)j * H + i) * C + c] = img[((size_t)i * W + j) * C + c];
}

/* Remove `count` vertical seams from an H x W image, recomputing the full energy before every
 * seam. The current image is in `buf` (capacity H*W*C), the result ends in `buf` with width
 * W-count. seam_log (nullable) receives count*H entries. */
static void carve_vertical(uint8_t *buf, uint8_t *tmp, int H, int W, int C, int count, int32_t *seam_log,
                           int64_t *cost_log) {
  uint16_t *e = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)H * W);
  int32_t *seam = (int32_t *)malloc(sizeof(int32_t) * H);
  for (int t = 0; t < count; ++t) {
    int w = W - t;
    orc_energy(buf, H, w, C, e);
    int64_t cost = orc_dp_seam(e, H, w, seam);
    if (seam_log) memcpy(seam_log + (size_t)t * H, seam, sizeof(int32_t) * H);
    if (cost_log) cost_log[t] = cost;
    orc_remove_seam(buf, H, w, C, seam, tmp);
    memcpy(buf, tmp, (size_t)H * (w - 1) * C);
  }
  free(e);
  free(seam);
}

/* The whole loop: (W - tw) vertical seams, then (H - th) horizontal seams via the transpose.
 * out receives th x tw x C. seam_log (nullable) receives (W-tw)*H vertical entries followed by
 * (H-th)*tw horizontal entries (in the transposed frame). Returns 0, or -1 on bad arguments. */
int orc_carve(const uint8_t *img, int H, int W, int C, int tw, int th, uint8_t *out, int32_t *seam_log,
              int64_t *cost_log) {
  if (H < 1 || W < 1 || C < 1 || tw < 1 || th < 1 || tw > W || th > H) return -1;
  size_t n = (size_t)H * W * C;
  uint8_t *buf = (uint8_t *)malloc(n);
  uint8_t *tmp = (uint8_t *)malloc(n);
  memcpy(buf, img, n);
  int nv = W - tw, nh = H - th;
  carve_vertical(buf, tmp, H, W, C, nv, seam_log, cost_log);
  if (nh > 0) {
    orc_transpose(buf, H, tw, C, tmp);                 /* now tw rows x H columns */
    memcpy(buf, tmp, (size_t)H * tw * C);
    carve_vertical(buf, tmp, tw, H, C, nh, seam_log ? seam_log + (size_t)nv * H : NULL,
                   cost_log ? cost_log + nv : NULL);
    orc_transpose(buf, tw, th, C, out);                /* back to th rows x tw columns */
  } else {
    memcpy(out, buf, (size_t)H * tw * C);
  }
  free(buf);
  free(tmp);
  return 0;
}

/* ---- seam insertion (reading R9) ----
 * out receives H x tw x C with tw = W + k; cols (nullable) receives the k mapped input columns of
 * every row, seam by seam (k*H entries). Returns 0, or -1 on bad arguments. */
int orc_enlarge(const uint8_t *img, int H, int W, int C, int tw, uint8_t *out, int32_t *cols) {
  const int k = tw - W;
  if (H < 1 || W < 1 || C < 1 || k < 1 || k > W - 1) return -1;
  size_t n = (size_t)H * W * C;
  uint8_t *buf = (uint8_t *)malloc(n);
  uint8_t *tmp = (uint8_t *)malloc(n);
  int32_t *log = (int32_t *)malloc(sizeof(int32_t) * (size_t)k * H);
  int *idx = (int *)malloc(sizeof(int) * W);
  uint8_t *dup = (uint8_t *)malloc(W);
  memcpy(buf, img, n);
  carve_vertical(buf, tmp, H, W, C, k, log, NULL);   /* the k seams, each in its own image's columns */
  for (int i = 0; i < H; ++i) {
    /* input column of every current column, updated by deleting each seam's entry in turn */
    for (int j = 0; j < W; ++j) idx[j] = j;
    memset(dup, 0, W);
    for (int t = 0; t < k; ++t) {
      int c = log[(size_t)t * H + i];
      int src = idx[c];
      dup[src] = 1;
      if (cols) cols[(size_t)t * H + i] = src;
      memmove(idx + c, idx + c + 1, sizeof(int) * (size_t)(W - t - 1 - c));
    }
    const uint8_t *row = img + (size_t)i * W * C;
    uint8_t *o = out + (size_t)i * tw * C;
    int q = 0;
    for (int j = 0; j < W; ++j) {
      for (int ch = 0; ch < C; ++ch) o[(size_t)q * C + ch] = row[(size_t)j * C + ch];
      ++q;
      if (dup[j]) {
        int jr = clampi(j + 1, 0, W - 1);
        for (int ch = 0; ch < C; ++ch)
          o[(size_t)q * C + ch] = (uint8_t)(((int)row[(size_t)j * C + ch] + (int)row[(size_t)jr * C + ch] + 1) / 2);
        ++q;
      }
    }
  }
  free(buf);
  free(tmp);
  free(log);
  free(idx);
  free(dup);
  return 0;
}

/* ---- forward energy (reading R10) ----
 * Three planes of H x W: CU, DL, DR (zero where the pair does not exist). */
void orc_forward_costs(const uint8_t *img, int H, int W, int C, uint16_t *cu, uint16_t *dl, uint16_t *dr) {
  for (int i = 0; i < H; ++i) {
    for (int j = 0; j < W; ++j) {
      int u = 0, l = 0, r = 0;
      for (int c = 0; c < C; ++c) {
        if (j >= 1 && j + 1 < W)
          u += absi((int)img[((size_t)i * W + j + 1) * C + c] - (int)img[((size_t)i * W + j - 1) * C + c]);
        if (i >= 1 && j >= 1)
          l += absi((int)img[((size_t)(i - 1) * W + j) * C + c] - (int)img[((size_t)i * W + j - 1) * C + c]);
        if (i >= 1 && j + 1 < W)
          r += absi((int)img[((size_t)(i - 1) * W + j) * C + c] - (int)img[((size_t)i * W + j + 1) * C + c]);
      }
      cu[(size_t)i * W + j] = (uint16_t)u;
      dl[(size_t)i * W + j] = (uint16_t)l;
      dr[(size_t)i * W + j] = (uint16_t)r;
    }
  }
}

/* Algorithm 3 with the forward costs: M(0,j) = CU(0,j); M(i,j) = CU(i,j) + min over in-range
 * j' in (j-1, j, j+1) of M(i-1,j') + (DL(i,j) if j' = j-1, 0 if j' = j, DR(i,j) if j' = j+1),
 * the leftmost candidate winning ties; backtrack and last-row argmin as R4, R5. */
int64_t orc_dp_seam_forward(const uint16_t *cu, const uint16_t *dl, const uint16_t *dr, int H, int W, int32_t *seam) {
  int64_t *M = (int64_t *)malloc(sizeof(int64_t) * (size_t)H * W);
  int32_t *B = (int32_t *)malloc(sizeof(int32_t) * (size_t)H * W);
  for (int j = 0; j < W; ++j) { M[j] = cu[j]; B[j] = -1; }
  for (int i = 1; i < H; ++i) {
    for (int j = 0; j < W; ++j) {
      int best = -1;
      int64_t bestv = 0;
      for (int jp = j - 1; jp <= j + 1; ++jp) {
        if (jp < 0 || jp >= W) continue;
        int64_t v = M[(size_t)(i - 1) * W + jp];
        if (jp == j - 1) v += dl[(size_t)i * W + j];
        if (jp == j + 1) v += dr[(size_t)i * W + j];
        if (best < 0 || v < bestv) { best = jp; bestv = v; }
      }
      B[(size_t)i * W + j] = best;
      M[(size_t)i * W + j] = (int64_t)cu[(size_t)i * W + j] + bestv;
    }
  }
  int jstar = 0;
  for (int j = 1; j < W; ++j)
    if (M[(size_t)(H - 1) * W + j] < M[(size_t)(H - 1) * W + jstar]) jstar = j;
  int64_t cost = M[(size_t)(H - 1) * W + jstar];
  seam[H - 1] = jstar;
  for (int i = H - 1; i >= 1; --i) seam[i - 1] = B[(size_t)i * W + seam[i]];
  free(M);
  free(B);
  return cost;
}

/* The full loop with forward energy: (W - tw) vertical seams, then (H - th) horizontal seams on the
 * transposed image, the forward costs recomputed from the current image before every seam. */
static void carve_vertical_forward(uint8_t *buf, uint8_t *tmp, int H, int W, int C, int count, int32_t *seam_log,
                                   int64_t *cost_log) {
  size_t n = (size_t)H * W;
  uint16_t *cu = (uint16_t *)malloc(sizeof(uint16_t) * n);
  uint16_t *dl = (uint16_t *)malloc(sizeof(uint16_t) * n);
  uint16_t *dr = (uint16_t *)malloc(sizeof(uint16_t) * n);
  int32_t *seam = (int32_t *)malloc(sizeof(int32_t) * H);
  for (int t = 0; t < count; ++t) {
    int w = W - t;
    orc_forward_costs(buf, H, w, C, cu, dl, dr);
    int64_t cost = orc_dp_seam_forward(cu, dl, dr, H, w, seam);
    if (seam_log) memcpy(seam_log + (size_t)t * H, seam, sizeof(int32_t) * H);
    if (cost_log) cost_log[t] = cost;
    orc_remove_seam(buf, H, w, C, seam, tmp);
    memcpy(buf, tmp, (size_t)H * (w - 1) * C);
  }
  free(cu);
  free(dl);
  free(dr);
  free(seam);
}

int orc_carve_forward(const uint8_t *img, int H, int W, int C, int tw, int th, uint8_t *out, int32_t *seam_log,
                      int64_t *cost_log) {
  if (H < 1 || W < 1 || C < 1 || tw < 1 || th < 1 || tw > W || th > H) return -1;
  size_t n = (size_t)H * W * C;
  uint8_t *buf = (uint8_t *)malloc(n);
  uint8_t *tmp = (uint8_t *)malloc(n);
  memcpy(buf, img, n);
  int nv = W - tw, nh = H - th;
  carve_vertical_forward(buf, tmp, H, W, C, nv, seam_log, cost_log);
  if (nh > 0) {
    orc_transpose(buf, H, tw, C, tmp);
    memcpy(buf, tmp, (size_t)H * tw * C);
    carve_vertical_forward(buf, tmp, tw, H, C, nh, seam_log ? seam_log + (size_t)nv * H : NULL,
                           cost_log ? cost_log + nv : NULL);
    orc_transpose(buf, tw, th, C, out);
  } else {
    memcpy(out, buf, (size_t)H * tw * C);
  }
  free(buf);
  free(tmp);
  return 0;
}
