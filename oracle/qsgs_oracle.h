/*
 * qsgs_oracle.h -- CPU oracle for the LIETS QSGS growth loop.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this code; the product library
 * never links, loads or calls it, and it shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * The oracle is a plain, slow, single-threaded statement of the method of
 * arXiv 2602.11734 (Wang & Al Kobaisi, "Ultra-Fast 3D Porous Media
 * Generation: a GPU-Accelerated List-Indexed Explicit Time-Stepping QSGS
 * Algorithm"): Bernoulli seeding (Sec. 2.1 step 2), diamond seed spacing
 * (Sec. 2.3, Fig. 1 D), the active front (Sec. 2.3 step 2), list-based
 * directional growth (Sec. 2.3 step 3, Algorithm 3), the front update
 * (Sec. 2.3 step 4) and the volume-fraction law of Eq. 1.  Each function in
 * qsgs_oracle.c cites the passage it follows.
 */
#ifndef QSGS_ORACLE_H
#define QSGS_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Generation parameters (the problem statement of Sec. 2.1 / Sec. 3.2). */
typedef struct {
  uint32_t nx, ny, nz;          /* grid dims, voxel v = x + nx*(y + ny*z)   */
  double cd;                    /* seed (core) probability c_d, in [0,1]    */
  double g_face;                /* G_ref of the 6 face directions           */
  double g_edge;                /* G_ref of the 12 edge directions          */
  double g_corner;              /* G_ref of the 8 corner directions         */
  uint32_t spacing_s;           /* minimum L1 distance between seeds        */
  double target_solid_fraction; /* phi_s                                    */
  uint64_t target_count;        /* Nt; 0 = derive from phi_s                */
  uint64_t seed;                /* RNG key                                  */
  uint32_t max_steps;           /* 0 = unlimited                            */
  uint32_t periodic;            /* 1: periodic domain (R11), each dim >= 3  */
  const uint8_t* blocked;       /* labels of earlier phases (R12): 0 = still
                                   unassigned, m >= 1 = cell of phase m;
                                   NULL: none                                */
  const double* inter;          /* R13: inter[3 (m - 1) + k] = interaction
                                   probability I^{n,m} of class k (face,
                                   edge, corner) for m = 1 .. n_labels; NULL
                                   or 0: phase m's cells are never entered  */
  uint32_t n_labels;            /* entries (labels) of inter                */
} oq_params;

typedef struct {
  uint32_t t;                   /* step index                               */
  uint64_t solid_before;        /* c_t                                      */
  uint64_t front;               /* |A_t|                                    */
  uint64_t claimed;             /* |New_t| before the final trim            */
  uint64_t thr[3];              /* Eq. 1 thresholds (face, edge, corner)    */
} oq_step_log;

typedef struct {
  uint64_t solid_count;         /* final c                                  */
  uint64_t target_count;        /* Nt                                       */
  uint64_t front_size;          /* |A| after the last step                  */
  uint64_t n_candidates;        /* Bernoulli candidates                     */
  uint64_t n_accepted;          /* seeds placed (after spacing and the cap) */
  uint32_t steps;               /* growth steps executed                    */
  int32_t status;               /* OQ_DONE / OQ_STALLED / OQ_MAX_STEPS      */
} oq_summary;

enum { OQ_DONE = 0, OQ_STALLED = 1, OQ_MAX_STEPS = 2 };
enum { OQ_ERR_INVALID = -1, OQ_ERR_NOMEM = -2 };

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void oq_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The 26 directions in canonical order: d=0..5 faces, 6..17 edges, 18..25
 * corners; within a class lexicographic in (dz, dy, dx).  dirs[3*d+0..2] =
 * (dx, dy, dz).  class_of[d] = 0 face, 1 edge, 2 corner. */
void oq_directions(int32_t dirs[78], int32_t class_of[26]);

/* Integer forms of the parameters: Nt, T_seed = floor(cd 2^32) and
 * T_ref[k] = floor(G_k 2^32).  Returns 0 or OQ_ERR_INVALID. */
int oq_targets(const oq_params* p, uint64_t* nt, uint64_t* t_seed, uint64_t t_ref[3]);

/* Eq. 1 threshold for solid count c: min(2^32, floor(t_ref (20 nt - 19 c) / nt)). */
uint64_t oq_threshold(uint64_t t_ref, uint64_t nt, uint64_t c);

/* Bernoulli candidates in ascending index; returns their number (writes at
 * most cap entries). */
uint64_t oq_seed_candidates(const oq_params* p, uint32_t* out, uint64_t cap);

/* Diamond spacing over an ascending candidate list: accepted[i] = 1 if kept. */
int oq_spacing(const oq_params* p, const uint32_t* cand, uint64_t n, uint8_t* accepted);

/* Active front of a phase map: solid voxels with a void in-domain
 * 26-neighbour, ascending; returns its size. */
uint64_t oq_front(const oq_params* p, const uint8_t* phase, uint32_t* out);

/* One full realization by the list-indexed scheme (Algorithm 3).
 * phase: N bytes written (1 solid, 0 void).  log may be NULL. */
int oq_run(const oq_params* p, uint8_t* phase, oq_step_log* log, uint32_t log_cap,
           oq_summary* out);

/* The same realization by the full-field synchronous sweep of Algorithm 2
 * (every solid voxel draws for every direction).  Test comparator only. */
int oq_run_fullfield(const oq_params* p, uint8_t* phase, oq_summary* out);

#ifdef __cplusplus
}
#endif
#endif /* QSGS_ORACLE_H */
