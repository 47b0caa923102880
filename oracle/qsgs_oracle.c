/*
 * qsgs_oracle.c -- CPU oracle for the LIETS QSGS growth loop.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product library.  Shares
 * no code with the CUDA path.
 *
 * Plain single-threaded C, written for a reader checking it against the
 * paper (arXiv 2602.11734).  Readings taken where the paper is silent or
 * ambiguous (each is also listed in the design notes):
 *
 *   R1  Random numbers.  The paper draws "an independent random number in
 *       (0,1)" per candidate (Sec. 2.3 step 3) from an unnamed generator.
 *       Here every draw is one 32-bit word of Philox4x32-10 (Salmon et al.,
 *       SC'11) keyed by the 64-bit realization seed:
 *         seeding draw of voxel v      : word v&3 of ctr (lo(v>>2), hi(v>>2), 0xFFFFFFFF, 0x100)
 *         growth draw of source a, step t, direction d, the r-th target of
 *         d's class c among a's targets at the start of step t (r counted
 *         in the direction order of R4):
 *                                      : word r&3 of ctr (lo(a), hi(a), t, 0x200 | B_c + r>>2)
 *       with B = 0 (faces), 2 (edges), 5 (corners).  A target is a neighbour
 *       inside the domain that is void (or, R13, may be entered) with a
 *       positive threshold; distinct attempts of a step use distinct words.
 *   R2  "u <= p" (Sec. 2.1 steps 2-3) and "rand < G" (Algorithms 1-3) are
 *       both read as r < floor(p 2^32) on the 32-bit word r, so the
 *       probability is exactly floor(p 2^32) / 2^32.
 *   R3  Eq. 1 with phi_a = c/N and phi_s = Nt/N gives the factor
 *       (20 Nt - 19 c) / Nt; it is evaluated once per step, before the step,
 *       in exact integers, and the threshold is clamped at 2^32.
 *   R4  Directions: the 26 neighbours (6 face, 12 edge, 8 corner) with one
 *       reference probability per class.
 *   R5  Front update: A_{t+1} = prune(A_t U New_t) (Sec. 1 and Sec. 2.3
 *       "appended"), not prune(New_t) alone (Algorithm 3 read literally).
 *   R6  Non-periodic domain: neighbours outside the grid are neither
 *       candidates (Algorithm 3, "inside domain") nor void.
 *   R12 Later growing phases (Sec. 2.1 step 4, independent discrete
 *       phases): a phase is generated "on the still unassigned cells" --
 *       cells of earlier phases (blocked) are never seeds, never void
 *       targets and never count as void neighbours; seeding, spacing, Eq. 1
 *       (phi_a = c/N over the whole domain) and the trim are otherwise those
 *       of the first phase.
 *   R13 Interacting phases (Sec. 2.1 step 4, second case): the phase being
 *       generated (n) grows into a neighbour that belongs to an earlier
 *       phase m with the interaction probability I^{n,m} of the direction's
 *       class, a constant (Eq. 1 scales the growth probabilities G only);
 *       a cell so entered becomes phase n's and counts towards its target,
 *       and the draw of such an attempt is the same keyed word as for a
 *       void target.  Unassigned cells are grown into with the Eq. 1
 *       probabilities as before.  A voxel of phase n is active (front) if
 *       it has a void neighbour or a neighbour of a phase m with a positive
 *       I^{n,m} for that direction's class.  Seeds are only placed on
 *       unassigned cells.  With every I = 0 this is R12.
 *   R11 Periodic option (the roll of Sec. 2.2 and Algorithm 2): with
 *       periodic = 1 the domain is a torus -- neighbours and the spacing
 *       distance wrap around every axis -- and every dimension must be at
 *       least 3, so that the 26 neighbours of a voxel are distinct.
 *   R7  Seed spacing: candidates are visited in ascending index; one is kept
 *       iff it lies outside the diamond (L1 ball of radius s-1, i.e. s-1
 *       dilations with the 6-connected kernel, Sec. 2.3 and Fig. 1 D) of
 *       every seed kept before it.  s <= 1 keeps all candidates.
 *   R8  Exact target: the loop of Algorithm 3 overshoots phi_s; here, if
 *       c_t + |New_t| > Nt, only the Nt - c_t lowest-index voxels of New_t
 *       are kept.  If the seeds alone exceed Nt, the Nt lowest are kept.
 *   R9  Nt = target_count if given, else floor(phi_s N + 0.5) in IEEE double.
 *   R10 Exits, tested in this order before every step: c >= Nt (done);
 *       t >= max_steps (step limit); no (source, direction) pair with a void
 *       in-domain target (or, R13, an enterable cell of an earlier phase)
 *       and a positive threshold (stalled -- the grid can never change
 *       again; an empty front is the special case).  A stalled step is not
 *       counted.
 */
#include "qsgs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11, Sec. 4.2 and Table 2): ten rounds of two 32x32  */
/* -> 64-bit products, the key bumped by a Weyl sequence between rounds.    */
/* ---------------------------------------------------------------------- */
void oq_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* Weyl key bumps    */
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * x0;
    uint64_t p1 = (uint64_t)M1 * x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0; k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ---------------------------------------------------------------------- */
/* Directions (R4): enumerate {-1,0,1}^3 \ 0 with dz slowest and dx fastest, */
/* then list faces, edges, corners, each in that enumeration order.         */
/* ---------------------------------------------------------------------- */
void oq_directions(int32_t dirs[78], int32_t class_of[26]) {
  int n = 0;
  for (int cls = 0; cls < 3; ++cls)
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int nonzero = (dx != 0) + (dy != 0) + (dz != 0);
          if (nonzero != cls + 1) continue;
          dirs[3 * n + 0] = dx;
          dirs[3 * n + 1] = dy;
          dirs[3 * n + 2] = dz;
          class_of[n] = cls;
          ++n;
        }
}

static uint64_t grid_size(const oq_params* p) {
  return (uint64_t)p->nx * (uint64_t)p->ny * (uint64_t)p->nz;
}

/* A cell of an earlier phase (R12). */
static int blocked(const oq_params* p, uint64_t v) { return p->blocked && p->blocked[v]; }

/* R13: threshold floor(I^{n,m} 2^32) of entering the cell v of an earlier
 * phase m along a direction of class k; 0 when phase m is not entered. */
static uint64_t inter_threshold(const oq_params* p, uint64_t v, int k) {
  const uint32_t m = p->blocked ? p->blocked[v] : 0u;
  if (m == 0 || !p->inter || m > p->n_labels) return 0;
  const double prob = p->inter[3 * (m - 1) + (uint32_t)k];
  if (!(prob > 0.0)) return 0;
  return (uint64_t)floor((prob < 1.0 ? prob : 1.0) * 4294967296.0);
}

/* R2 / R9: integer forms of the parameters. */
int oq_targets(const oq_params* p, uint64_t* nt, uint64_t* t_seed, uint64_t t_ref[3]) {
  const double two32 = 4294967296.0;
  uint64_t n = grid_size(p);
  if (p->nx == 0 || p->ny == 0 || p->nz == 0 || n >= 4294967296ull) return OQ_ERR_INVALID;
  if (p->periodic > 1) return OQ_ERR_INVALID;
  if (p->periodic && (p->nx < 3 || p->ny < 3 || p->nz < 3)) return OQ_ERR_INVALID;  /* R11 */
  if (!(p->cd >= 0.0 && p->cd <= 1.0)) return OQ_ERR_INVALID;
  if (!(p->g_face >= 0.0 && p->g_face <= 1.0)) return OQ_ERR_INVALID;
  if (!(p->g_edge >= 0.0 && p->g_edge <= 1.0)) return OQ_ERR_INVALID;
  if (!(p->g_corner >= 0.0 && p->g_corner <= 1.0)) return OQ_ERR_INVALID;
  uint64_t target;
  if (p->target_count != 0) {
    target = p->target_count;
  } else {
    if (!(p->target_solid_fraction >= 0.0 && p->target_solid_fraction <= 1.0)) return OQ_ERR_INVALID;
    target = (uint64_t)floor(p->target_solid_fraction * (double)n + 0.5);
  }
  if (target > n) return OQ_ERR_INVALID;
  *nt = target;
  *t_seed = (uint64_t)floor(p->cd * two32);
  t_ref[0] = (uint64_t)floor(p->g_face * two32);
  t_ref[1] = (uint64_t)floor(p->g_edge * two32);
  t_ref[2] = (uint64_t)floor(p->g_corner * two32);
  return 0;
}

/* Eq. 1: G(phi_a) = G_ref (phi_s - 0.95 phi_a) / (0.05 phi_s), with
 * phi_a = c/N, phi_s = nt/N, i.e. G_ref (20 nt - 19 c) / nt (R3). */
uint64_t oq_threshold(uint64_t t_ref, uint64_t nt, uint64_t c) {
  const uint64_t two32 = 4294967296ull;
  if (nt == 0) return t_ref < two32 ? t_ref : two32;
  __int128 num = (__int128)20 * nt - (__int128)19 * c;
  if (num <= 0) return 0;
  unsigned __int128 prod = (unsigned __int128)t_ref * (unsigned __int128)num;
  unsigned __int128 q = prod / nt;
  return q > two32 ? two32 : (uint64_t)q;
}

/* Sec. 2.1 step 2: every cell draws a uniform number; it becomes a core
 * (seed candidate) if the number does not exceed c_d (R1, R2). */
uint64_t oq_seed_candidates(const oq_params* p, uint32_t* out, uint64_t cap) {
  uint64_t nt, t_seed, t_ref[3];
  if (oq_targets(p, &nt, &t_seed, t_ref) != 0) return 0;
  uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
  uint64_t n = grid_size(p), count = 0;
  for (uint64_t v = 0; v < n; ++v) {
    uint64_t group = v >> 2;
    uint32_t ctr[4] = {(uint32_t)group, (uint32_t)(group >> 32), 0xFFFFFFFFu, 0x100u};
    uint32_t r[4];
    oq_philox4x32_10(ctr, key, r);
    if ((uint64_t)r[v & 3] < t_seed && !blocked(p, v)) {
      if (count < cap) out[count] = (uint32_t)v;
      ++count;
    }
  }
  return count;
}

/* Sec. 2.3 and Fig. 1 D, reading R7: visit candidates in ascending index;
 * keep one unless an earlier kept seed's diamond (every voxel within L1
 * distance s-1, the result of s-1 dilations with the 6-connected kernel)
 * already covers it; then stamp the kept seed's own diamond. */
int oq_spacing(const oq_params* p, const uint32_t* cand, uint64_t n, uint8_t* accepted) {
  if (p->spacing_s <= 1) {
    for (uint64_t i = 0; i < n; ++i) accepted[i] = 1;
    return 0;
  }
  const int64_t nx = p->nx, ny = p->ny, nz = p->nz;
  const int64_t r = (int64_t)p->spacing_s - 1;
  uint8_t* covered = (uint8_t*)calloc((size_t)(nx * ny * nz), 1);
  if (!covered) return OQ_ERR_NOMEM;
  for (uint64_t i = 0; i < n; ++i) {
    int64_t v = cand[i];
    if (covered[v]) { accepted[i] = 0; continue; }
    accepted[i] = 1;
    int64_t x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
    for (int64_t dz = -r; dz <= r; ++dz) {
      int64_t zz = z + dz;
      if (p->periodic) zz = ((zz % nz) + nz) % nz; /* R11: the diamond wraps */
      else if (zz < 0 || zz >= nz) continue;
      int64_t rz = r - llabs(dz);
      for (int64_t dy = -rz; dy <= rz; ++dy) {
        int64_t yy = y + dy;
        if (p->periodic) yy = ((yy % ny) + ny) % ny;
        else if (yy < 0 || yy >= ny) continue;
        int64_t ry = rz - llabs(dy);
        for (int64_t dx = -ry; dx <= ry; ++dx) {
          int64_t xx = x + dx;
          if (p->periodic) xx = ((xx % nx) + nx) % nx;
          else if (xx < 0 || xx >= nx) continue;
          covered[xx + nx * (yy + ny * zz)] = 1;
        }
      }
    }
  }
  free(covered);
  return 0;
}

/* Neighbour q of voxel v in direction (dx,dy,dz) if inside the domain (R6);
 * on the torus every neighbour exists (R11). */
static int neighbour(const oq_params* p, uint64_t v, int dx, int dy, int dz, uint64_t* q) {
  int64_t nx = p->nx, ny = p->ny, nz = p->nz;
  int64_t x = (int64_t)(v % (uint64_t)nx);
  int64_t y = (int64_t)((v / (uint64_t)nx) % (uint64_t)ny);
  int64_t z = (int64_t)(v / ((uint64_t)nx * (uint64_t)ny));
  x += dx; y += dy; z += dz;
  if (p->periodic) {
    x = (x + nx) % nx;
    y = (y + ny) % ny;
    z = (z + nz) % nz;
  }
  if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) return 0;
  *q = (uint64_t)(x + nx * (y + ny * z));
  return 1;
}

/* "Solid cells which have at least one neighboring void cell" (Sec. 2.3
 * step 2), over the same 26 directions as growth; with interacting phases
 * (R13) a neighbour of a phase that may be entered along that direction
 * counts as well. */
static int has_void_neighbour(const oq_params* p, const uint8_t* phase, uint64_t v,
                              const int32_t dirs[78], const int32_t cls[26]) {
  for (int d = 0; d < 26; ++d) {
    uint64_t q;
    if (!neighbour(p, v, dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2], &q) || phase[q] != 0)
      continue;
    if (!blocked(p, q) || inter_threshold(p, q, cls[d]) > 0) return 1;
  }
  return 0;
}

/* R1 (growth draws): the targets of a source at the start of a step, as a
 * 26-bit mask over the directions -- neighbours inside the domain that are
 * void with a positive threshold of their class, or (R13) cells of an
 * earlier phase that may be entered along that direction. */
static uint32_t target_mask(const oq_params* p, const uint8_t* phase, uint64_t a,
                            const int32_t dirs[78], const int32_t cls[26], const uint64_t thr[3]) {
  uint32_t m = 0;
  for (int d = 0; d < 26; ++d) {
    uint64_t q;
    if (!neighbour(p, a, dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2], &q) || phase[q] != 0)
      continue;
    const uint64_t th = blocked(p, q) ? inter_threshold(p, q, cls[d]) : thr[cls[d]];
    if (th > 0) m |= 1u << d;
  }
  return m;
}

static int count_bits(uint32_t m) {
  int n = 0;
  for (; m; m &= m - 1) ++n;
  return n;
}

/* R1 (growth draws): the attempt of source a along direction d at step t is
 * the r-th target of d's class (r counted over the class's directions in
 * canonical order, among the targets of the start of the step); it takes
 * word r & 3 of the Philox block with counter (a lo, a hi, t, 0x200 | b),
 * b = B_class + (r >> 2), B = 0 (faces: blocks 0, 1), 2 (edges: 2, 3, 4), 5
 * (corners: 5, 6).  Distinct attempts of a step thus use distinct words. */
static uint32_t growth_draw(uint64_t a, uint32_t t, uint32_t targets, int d, int klass,
                            const uint32_t key[2]) {
  static const uint32_t class_bits[3] = {0x3Fu, 0x3FFC0u, 0x3FC0000u};
  static const uint32_t first_block[3] = {0u, 2u, 5u};
  const int r = count_bits(targets & class_bits[klass] & ((1u << d) - 1u));
  const uint32_t ctr[4] = {(uint32_t)a, (uint32_t)(a >> 32), t,
                           0x200u | (first_block[klass] + (uint32_t)(r >> 2))};
  uint32_t out[4];
  oq_philox4x32_10(ctr, key, out);
  return out[r & 3];
}

uint64_t oq_front(const oq_params* p, const uint8_t* phase, uint32_t* out) {
  int32_t dirs[78], cls[26];
  oq_directions(dirs, cls);
  uint64_t n = grid_size(p), k = 0;
  for (uint64_t v = 0; v < n; ++v)
    if (phase[v] && has_void_neighbour(p, phase, v, dirs, cls)) out[k++] = (uint32_t)v;
  return k;
}

static int cmp_u32(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return (x > y) - (x < y);
}

/* Seeding, spacing and the cap on the seed count (Sec. 2.1 step 2, Sec. 2.3
 * step 1, R7, R8).  Writes the seeds into phase (zeroed first); returns the
 * number placed, or a negative error. */
static int64_t place_seeds(const oq_params* p, uint64_t nt, uint8_t* phase, oq_summary* out) {
  uint64_t n = grid_size(p);
  memset(phase, 0, (size_t)n);
  uint64_t n_cand = oq_seed_candidates(p, NULL, 0);
  uint32_t* cand = (uint32_t*)malloc((size_t)(n_cand ? n_cand : 1) * sizeof(uint32_t));
  uint8_t* acc = (uint8_t*)malloc((size_t)(n_cand ? n_cand : 1));
  if (!cand || !acc) { free(cand); free(acc); return OQ_ERR_NOMEM; }
  oq_seed_candidates(p, cand, n_cand);
  int rc = oq_spacing(p, cand, n_cand, acc);
  if (rc != 0) { free(cand); free(acc); return rc; }
  uint64_t placed = 0;
  for (uint64_t i = 0; i < n_cand && placed < nt; ++i)
    if (acc[i]) { phase[cand[i]] = 1; ++placed; }
  out->n_candidates = n_cand;
  out->n_accepted = placed;
  free(cand);
  free(acc);
  return (int64_t)placed;
}

/* Algorithm 3 (Sec. 2.3 steps 1-5). */
int oq_run(const oq_params* p, uint8_t* phase, oq_step_log* log, uint32_t log_cap,
           oq_summary* out) {
  uint64_t nt, t_seed, t_ref[3];
  memset(out, 0, sizeof(*out));
  int rc = oq_targets(p, &nt, &t_seed, t_ref);
  if (rc != 0) return rc;
  int32_t dirs[78], cls[26];
  oq_directions(dirs, cls);
  uint64_t n = grid_size(p);
  uint32_t max_steps = p->max_steps ? p->max_steps : 0xFFFFFFFFu;
  uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};

  int64_t placed = place_seeds(p, nt, phase, out);
  if (placed < 0) return (int)placed;
  uint64_t c = (uint64_t)placed; /* phi_a = c / N */

  uint32_t* A = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  uint32_t* A_new = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  uint32_t* merged = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  uint32_t* T = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));  /* targets of A[i] */
  if (!A || !A_new || !merged || !T) {
    free(A); free(A_new); free(merged); free(T);
    return OQ_ERR_NOMEM;
  }

  /* Algorithm 3 starts from the active set: solids with a void neighbour
   * (step 2 of Sec. 2.3). */
  uint64_t a_n = oq_front(p, phase, A);
  uint32_t t = 0;
  int32_t status;
  /* Loop while phi_a < phi_s and A is not empty (R10 for the order of the
   * three exits). */
  for (;;) {
    if (c >= nt) { status = OQ_DONE; break; }
    if (t >= max_steps) { status = OQ_MAX_STEPS; break; }
    uint64_t thr[3];
    for (int k = 0; k < 3; ++k) thr[k] = oq_threshold(t_ref[k], nt, c); /* Eq. 1 */
    uint64_t new_n = 0, live = 0;  /* A_new starts empty each step */
    /* The targets of every front voxel at the start of the step (the draws
     * are located by rank among them, R1). */
    for (uint64_t i = 0; i < a_n; ++i) T[i] = target_mask(p, phase, A[i], dirs, cls, thr);
    for (int d = 0; d < 26; ++d) {   /* every direction of every front voxel */
      for (uint64_t i = 0; i < a_n; ++i) {
        uint64_t a = A[i], q;
        /* neighbours inside the domain that were void at the start of the
         * step -- or, with interacting phases (R13), cells of an earlier
         * phase -- with a positive threshold */
        if (!((T[i] >> d) & 1u)) continue;
        neighbour(p, a, dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2], &q);
        if (phase[q] != 0) continue;  /* claimed earlier in this step */
        const uint64_t th = blocked(p, q) ? inter_threshold(p, q, cls[d]) : thr[cls[d]];
        ++live;
        /* an independent draw for this (source, step, direction) */
        if ((uint64_t)growth_draw(a, t, T[i], d, cls[d], key) < th) {
          phase[q] = 1;  /* the void (or entered cell) becomes solid ... */
          A_new[new_n++] = (uint32_t)q;  /* ... and joins A_new */
        }
      }
    }
    /* No attempt with a positive probability: the grid is a fixed point
     * (an empty front is the special case A = {}). */
    if (live == 0) { status = OQ_STALLED; break; }
    if (log && t < log_cap) {
      log[t].t = t;
      log[t].solid_before = c;
      log[t].front = a_n;
      log[t].claimed = new_n;
      for (int k = 0; k < 3; ++k) log[t].thr[k] = thr[k];
    }
    /* The next front is prune(A U A_new) (R1) -- duplicates cannot occur;
     * A_new is sorted so that the exact-target trim (R8) keeps its lowest
     * indices. */
    qsort(A_new, (size_t)new_n, sizeof(uint32_t), cmp_u32);
    if (c + new_n > nt) {
      uint64_t keep = nt - c;
      for (uint64_t i = keep; i < new_n; ++i) phase[A_new[i]] = 0;
      new_n = keep;
    }
    c += new_n; /* phi_a of the updated phase array */
    uint64_t i = 0, j = 0, m = 0;
    while (i < a_n || j < new_n) {
      uint32_t v;
      if (j >= new_n || (i < a_n && A[i] < A_new[j])) v = A[i++];
      else v = A_new[j++];
      if (has_void_neighbour(p, phase, v, dirs, cls)) merged[m++] = v;
    }
    uint32_t* tmp = A; A = merged; merged = tmp;
    a_n = m;
    ++t;
  }
  out->solid_count = c;
  out->target_count = nt;
  out->front_size = a_n;
  out->steps = t;
  out->status = status;
  free(A);
  free(A_new);
  free(merged);
  free(T);
  return 0;
}

/* Algorithm 2 (Sec. 2.2), with the same draws as oq_run: each step every
 * solid cell of the start-of-step mask draws in every direction, and the
 * accepted neighbours are OR-ed into the phase array (non-periodic shift,
 * R6, or the periodic roll, R11).  Stops like Algorithm 3: target reached, no solid cell with a void
 * neighbour left, or the step limit. */
int oq_run_fullfield(const oq_params* p, uint8_t* phase, oq_summary* out) {
  uint64_t nt, t_seed, t_ref[3];
  memset(out, 0, sizeof(*out));
  int rc = oq_targets(p, &nt, &t_seed, t_ref);
  if (rc != 0) return rc;
  int32_t dirs[78], cls[26];
  oq_directions(dirs, cls);
  uint64_t n = grid_size(p);
  uint32_t max_steps = p->max_steps ? p->max_steps : 0xFFFFFFFFu;
  uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};

  int64_t placed = place_seeds(p, nt, phase, out);
  if (placed < 0) return (int)placed;
  uint64_t c = (uint64_t)placed;
  uint8_t* solid_mask = (uint8_t*)malloc((size_t)n);
  uint8_t* grown = (uint8_t*)malloc((size_t)n);
  uint32_t* T = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));  /* targets of each cell */
  if (!solid_mask || !grown || !T) {
    free(solid_mask); free(grown); free(T);
    return OQ_ERR_NOMEM;
  }

  uint32_t t = 0;
  int32_t status;
  for (;;) {
    if (c >= nt) { status = OQ_DONE; break; }
    if (t >= max_steps) { status = OQ_MAX_STEPS; break; }
    uint64_t thr[3];
    for (int k = 0; k < 3; ++k) thr[k] = oq_threshold(t_ref[k], nt, c);
    memcpy(solid_mask, phase, (size_t)n);
    memset(grown, 0, (size_t)n);
    uint64_t live = 0;
    /* the targets of every solid cell of the start-of-step mask (R1) */
    for (uint64_t a = 0; a < n; ++a)
      T[a] = solid_mask[a] ? target_mask(p, solid_mask, a, dirs, cls, thr) : 0u;
    for (int d = 0; d < 26; ++d) {
      for (uint64_t a = 0; a < n; ++a) {
        if (!solid_mask[a] || !((T[a] >> d) & 1u)) continue;
        uint64_t q;
        /* a target: void, or (R13) a cell of an earlier phase */
        neighbour(p, a, dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2], &q);
        const uint64_t th = blocked(p, q) ? inter_threshold(p, q, cls[d]) : thr[cls[d]];
        ++live;
        if ((uint64_t)growth_draw(a, t, T[a], d, cls[d], key) >= th) continue;
        grown[q] = 1;
      }
    }
    if (live == 0) { status = OQ_STALLED; break; }
    uint64_t new_n = 0;
    for (uint64_t v = 0; v < n; ++v) new_n += grown[v];
    uint64_t keep = (c + new_n > nt) ? nt - c : new_n, kept = 0;
    for (uint64_t v = 0; v < n; ++v)
      if (grown[v]) {
        if (kept < keep) { phase[v] = 1; ++kept; }
      }
    c += kept;
    ++t;
  }
  uint64_t front = 0;
  for (uint64_t v = 0; v < n; ++v)
    if (phase[v] && has_void_neighbour(p, phase, v, dirs, cls)) ++front;
  out->solid_count = c;
  out->target_count = nt;
  out->front_size = front;
  out->steps = t;
  out->status = status;
  free(solid_mask);
  free(grown);
  free(T);
  return 0;
}
