/*
 * dsr_oracle.c -- plain, sequential CPU oracle for the generic-mode
 * data-sharing runtime.
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this library; the product path (the CUDA
 * library) never calls it, and the two share no code, header or helper.
 *
 * What it computes. OpenMP "parallel nested in target" semantics (Sec. 3.2
 * and Fig. "target-parallel" (b); Sec. 4): in each team one master thread
 * runs the sequential code block; locals that a nested parallel region
 * references are shared with the workers of that region by reference
 * (Sec. 5.1: master and workers follow the same reference, so each sees the
 * other's writes; master/worker accesses never race, worker/worker races
 * are the user's). The paper lowers those locals to a per-team stack in
 * shared memory (Sec. 5.3, "Shared memory stack") with a global-memory
 * safety net (Sec. 5.2, last paragraph; Sec. 7).
 *
 * The oracle is the plain definition of that: per team it runs the master's
 * code; every frame of shared locals is an ordinary heap buffer kept on a
 * LIFO list; every parallel region runs its workers tid = 0 .. nthreads-1
 * one after another, to completion, before the master resumes (the fork /
 * join of Sec. 4, Fig. "codegen-master" and "codegen-worker"). For a
 * race-free program this is the result of every schedule of the workers.
 *
 * Stack accounting (not placement-dependent results, but checked): each
 * push reserves its size rounded up to 16 bytes, in the shared-memory slab
 * if it still fits there, else in the team's overflow slab, else the push
 * fails with status OVERFLOW and the team unwinds. hwm = peak of reserved
 * bytes over both; spill = peak of overflow-slab bytes.
 *
 * Integer arithmetic is modulo 2^32. mix32 is the 32-bit finaliser of
 * MurmurHash3 (Austin Appleby, public domain), written from its published
 * description. Floating point: the FP32 sweep program's sums are kept two
 * ways: in double (fp64), with the sum of magnitudes for the error bound,
 * and as the fp32 sum itself, taken in index order with every addition
 * rounded to fp32 (the program's definition; this file is compiled with
 * -ffp-contract=off, and the sum has no multiply to contract anyway).
 *
 * The region programs (shared locals, sequential code, bodies) are defined
 * in the comments of each team_* function below; W = threads - 32 is the
 * number of workers and W' = max(W, 1) the width of every parallel region
 * (with no workers the master runs the region as a team of one). A region
 * may ask for fewer threads (the descriptor's width, 1 <= width <= W'): the
 * workers beyond it skip the body (Sec. 4, Fig. "codegen-worker", the
 * exec_status test); "width" below means that effective thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_OVERFLOW 2
#define ORC_ERR_LIFO 3

#define ORC_MAX_LEVELS 4   /* frame sizes a region descriptor carries */
#define ORC_STACK_CAP 16   /* frame-table entries per team */
#define ORC_WARP_CAP 32    /* frames of one warp's stack (one per lane) */

enum {
  PROG_PAPER_SCALARS = 1,
  PROG_PAPER_ARRAYS = 2,
  PROG_SCALARS = 3,
  PROG_NESTED = 4,
  PROG_SWEEP = 5,
  PROG_HETERO = 6,
  PROG_WORKERS = 7,
};

/* One region instance (64 bytes). */
typedef struct {
  uint32_t program;
  uint32_t teams;
  uint32_t threads;
  uint32_t depth;
  uint32_t frame_bytes[ORC_MAX_LEVELS];
  uint32_t width; /* threads of each parallel region; 0 = every worker */
  uint32_t param;
  uint32_t salt;
  uint32_t status_index;
  uint64_t image_offset;
  uint64_t out_offset;
} orc_region;

/* Per-team result record (32 bytes). */
typedef struct {
  int32_t status;
  uint32_t depth_final;
  uint32_t hwm_bytes;
  uint32_t spill_bytes;
  uint32_t chk[ORC_MAX_LEVELS];
} orc_team_status;

/* ------------------------------------------------------------------------ */
/* mix32: MurmurHash3 fmix32                                                */
/* ------------------------------------------------------------------------ */
uint32_t orc_mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

/* ------------------------------------------------------------------------ */
/* The team's LIFO stack of frames (Sec. 5.3 shared stack + Sec. 5.2 / 7     */
/* global safety net)                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint8_t *data;
  uint64_t footprint; /* bytes reserved on the stack (size rounded to 16) */
  int in_slab;
} orc_frame;

typedef struct {
  orc_frame f[ORC_WARP_CAP];
  uint32_t cap; /* frame-table entries: ORC_STACK_CAP, or ORC_WARP_CAP for a warp's stack */
  uint32_t depth;
  uint64_t slab_cap, ovf_cap;
  uint64_t slab_used, ovf_used;
  uint64_t hwm, spill_hwm;
  int32_t status;
} orc_stack;

static void stack_init(orc_stack *s, uint64_t slab_cap, uint64_t ovf_cap) {
  memset(s, 0, sizeof(*s));
  s->cap = ORC_STACK_CAP;
  s->slab_cap = slab_cap;
  s->ovf_cap = ovf_cap;
}

static uint8_t *push(orc_stack *s, uint32_t bytes) {
  uint64_t fp = ((uint64_t)bytes + 15u) & ~(uint64_t)15u;
  int in_slab;
  if (s->depth == s->cap) {
    s->status = ORC_ERR_OVERFLOW;
    return NULL;
  }
  if (s->slab_used + fp <= s->slab_cap) {
    in_slab = 1;
    s->slab_used += fp;
  } else if (s->ovf_used + fp <= s->ovf_cap) {
    in_slab = 0;
    s->ovf_used += fp;
  } else {
    s->status = ORC_ERR_OVERFLOW;
    return NULL;
  }
  orc_frame *f = &s->f[s->depth++];
  f->data = (uint8_t *)calloc(fp ? fp : 16, 1);
  f->footprint = fp;
  f->in_slab = in_slab;
  if (s->slab_used + s->ovf_used > s->hwm) s->hwm = s->slab_used + s->ovf_used;
  if (s->ovf_used > s->spill_hwm) s->spill_hwm = s->ovf_used;
  return f->data;
}

/* Pop `data`, which must be the top frame (LIFO). */
static int pop(orc_stack *s, uint8_t *data) {
  if (s->depth == 0 || s->f[s->depth - 1].data != data) {
    s->status = ORC_ERR_LIFO;
    return ORC_ERR_LIFO;
  }
  orc_frame *f = &s->f[--s->depth];
  if (f->in_slab)
    s->slab_used -= f->footprint;
  else
    s->ovf_used -= f->footprint;
  free(f->data);
  f->data = NULL;
  return ORC_OK;
}

static void unwind(orc_stack *s) {
  while (s->depth) pop(s, s->f[s->depth - 1].data);
}

static uint32_t ld32(const uint8_t *p) {
  uint32_t v;
  memcpy(&v, p, 4);
  return v;
}
static void st32(uint8_t *p, uint32_t v) { memcpy(p, &v, 4); }

static uint32_t team_width(const orc_region *d) {
  return d->threads > 32 ? d->threads - 32 : 1;
}
static uint32_t width(const orc_region *d) {
  return d->width ? d->width : team_width(d);
}

/* ------------------------------------------------------------------------ */
/* PX1: the paper's scalar-sharing program (Sec. 6.1, Fig. "Implicitly      */
/* sharing 8 variables"). Shared locals: int c[n] and the reference to the  */
/* mapped array a. Master: every c_i starts at 0, then c_i += i (the        */
/* listing's "c1 += 1 ... c7 += 7"). Parallel: a[team*W' + tid] += sum c_i.  */
/* ------------------------------------------------------------------------ */
static void team_paper_scalars(const orc_region *d, uint32_t team, uint8_t *out,
                               orc_stack *s) {
  uint32_t n = d->param, w = width(d);
  uint8_t *f = push(s, d->frame_bytes[0]);
  if (!f) return;
  uint32_t ptr_off = (4u * n + 7u) & ~7u;
  for (uint32_t i = 0; i < n; i++) st32(f + 4 * i, 0);
  for (uint32_t i = 0; i < n; i++) st32(f + 4 * i, ld32(f + 4 * i) + (i + 1));
  int32_t *a = (int32_t *)(out + d->out_offset);
  memcpy(f + ptr_off, &a, sizeof(a)); /* the reference to a (Sec. 5.1) */
  for (uint32_t tid = 0; tid < w; tid++) {
    int32_t *aref;
    memcpy(&aref, f + ptr_off, sizeof(aref));
    uint32_t sum = 0;
    for (uint32_t i = 0; i < n; i++) sum += ld32(f + 4 * i);
    uint32_t *slot = (uint32_t *)&aref[team * w + tid];
    *slot = *slot + sum;
  }
  pop(s, f);
}

/* ------------------------------------------------------------------------ */
/* PX2: the paper's array-sharing program (Sec. 6.1, Fig. "Implicitly       */
/* sharing an array"). Shared locals: k arrays int d_m[W']. Master: fills   */
/* every d_m[i] = 10. Parallel: a[team*W' + tid] += sum_m d_m[tid].          */
/* ------------------------------------------------------------------------ */
static void team_paper_arrays(const orc_region *d, uint32_t team, uint8_t *out,
                              orc_stack *s) {
  uint32_t k = d->param, w = width(d);
  uint8_t *f = push(s, d->frame_bytes[0]);
  if (!f) return;
  for (uint32_t m = 0; m < k; m++)
    for (uint32_t i = 0; i < w; i++) st32(f + 4 * (m * w + i), 10);
  uint32_t *a = (uint32_t *)(out + d->out_offset);
  for (uint32_t tid = 0; tid < w; tid++) {
    uint32_t sum = 0;
    for (uint32_t m = 0; m < k; m++) sum += ld32(f + 4 * (m * w + tid));
    a[team * w + tid] += sum;
  }
  pop(s, f);
}

/* ------------------------------------------------------------------------ */
/* P1 "scalars": R = param sequential regions per team. Region r: the master*/
/* pushes int32 s[4] = image[r][0..3]; parallel: out[(r*T + team)*W' + tid] */
/*    =                                                                     */
/* (s0*tid + s1) ^ ((s2 >> (tid & 7)) + s3)  (C precedence: + before ^).   */
/* ------------------------------------------------------------------------ */
static void team_scalars(const orc_region *d, uint32_t team, const uint8_t *img,
                         uint8_t *out, orc_stack *s) {
  uint32_t w = width(d);
  uint32_t *o = (uint32_t *)(out + d->out_offset);
  for (uint32_t r = 0; r < d->param; r++) {
    uint8_t *f = push(s, 16);
    if (!f) return;
    memcpy(f, img + d->image_offset + 16ull * r, 16);
    for (uint32_t tid = 0; tid < w; tid++) {
      uint32_t s0 = ld32(f), s1 = ld32(f + 4), s2 = ld32(f + 8), s3 = ld32(f + 12);
      o[((uint64_t)r * d->teams + team) * w + tid] =
          (s0 * tid + s1) ^ ((s2 >> (tid & 7u)) + s3);
    }
    pop(s, f);
  }
}

/* ------------------------------------------------------------------------ */
/* P2 "nested": D levels, each a master-side call with its own frame        */
/* F_k = { int32 s[16]; int32 arr[256] } and its own parallel region.        */
/* Level k = 1..D:                                                          */
/*   master: push F_k; F_k[i] = image[team][k-1][i] ^ mix32(team*8 + k);     */
/*           if k > 1: F_k.s[0] ^= F_{k-1}.s[15].                            */
/*   parallel, k < D: for i = tid; i < 256; i += W':                         */
/*           F_k.arr[i] = mix32(F_k.arr[i] + i)                              */
/*   parallel, k = D: for j = tid; j < E; j += W', e = team*E + j:           */
/*           out[e] = mix32(e ^ sum_{m=1..D} (F_m.arr[j&255] ^ F_m.s[j&15])) */
/*   master after the join, k < D: F_k.s[15] = sum_i F_k.arr[i].             */
/* Unwind k = D..1: chk[k-1] = F_k.s[15]; pop F_k.                          */
/* ------------------------------------------------------------------------ */
static void team_nested(const orc_region *d, uint32_t team, const uint8_t *img,
                        uint8_t *out, orc_stack *s, orc_team_status *st) {
  uint32_t w = width(d), D = d->depth, E = d->param;
  uint8_t *F[ORC_MAX_LEVELS] = {0};
  uint32_t *o = (uint32_t *)(out + d->out_offset);
  const uint8_t *timg = img + d->image_offset + (uint64_t)team * D * 1088u;
  for (uint32_t k = 1; k <= D; k++) {
    uint8_t *f = push(s, d->frame_bytes[k - 1]);
    if (!f) return;
    F[k - 1] = f;
    uint32_t key = orc_mix32(team * 8u + k);
    for (uint32_t i = 0; i < 272; i++) st32(f + 4 * i, ld32(timg + (k - 1) * 1088u + 4 * i) ^ key);
    if (k > 1) st32(f, ld32(f) ^ ld32(F[k - 2] + 4 * 15));
    for (uint32_t tid = 0; tid < w; tid++) {
      if (k < D) {
        for (uint32_t i = tid; i < 256; i += w) {
          uint8_t *p = f + 64 + 4 * i;
          st32(p, orc_mix32(ld32(p) + i));
        }
      } else {
        for (uint32_t j = tid; j < E; j += w) {
          uint32_t e = team * E + j, acc = 0;
          for (uint32_t m = 0; m < D; m++)
            acc += ld32(F[m] + 64 + 4 * (j & 255u)) ^ ld32(F[m] + 4 * (j & 15u));
          o[(uint64_t)team * E + j] = orc_mix32(e ^ acc);
        }
      }
    }
    if (k < D) {
      uint32_t sum = 0;
      for (uint32_t i = 0; i < 256; i++) sum += ld32(f + 64 + 4 * i);
      st32(f + 4 * 15, sum);
    }
  }
  for (uint32_t k = D; k >= 1; k--) {
    st->chk[k - 1] = ld32(F[k - 1] + 4 * 15);
    pop(s, F[k - 1]);
  }
}

/* ------------------------------------------------------------------------ */
/* P3 "sweep": one frame float arr[L], L = S/4. Master: arr = image[team].   */
/* Parallel: out[team*W' + tid] = arr[tid] + arr[tid+W'] + arr[tid+2W'] ... */
/* (index order, each addition rounded to fp32). The oracle keeps three     */
/* values per output slot: the sum and the sum of magnitudes (for the error */
/* bound) in double, and the fp32 sum as defined, widened to double: out is */
/* double[T][W'][3].                                                        */
/* ------------------------------------------------------------------------ */
static void team_sweep(const orc_region *d, uint32_t team, const uint8_t *img,
                       uint8_t *out, orc_stack *s) {
  uint32_t w = width(d), L = d->frame_bytes[0] / 4;
  uint8_t *f = push(s, d->frame_bytes[0]);
  if (!f) return;
  memcpy(f, img + d->image_offset + (uint64_t)team * L * 4, (size_t)L * 4);
  /* each 4-byte output slot of the product becomes 24 bytes here */
  double *o = (double *)(out + 6 * d->out_offset);
  for (uint32_t tid = 0; tid < w; tid++) {
    double sum = 0.0, mag = 0.0;
    float sum32 = 0.0f;
    for (uint32_t i = tid; i < L; i += w) {
      float x;
      memcpy(&x, f + 4ull * i, 4);
      sum += (double)x;
      mag += x < 0 ? -(double)x : (double)x;
      sum32 = sum32 + x;
    }
    o[3 * ((uint64_t)team * w + tid)] = sum;
    o[3 * ((uint64_t)team * w + tid) + 1] = mag;
    o[3 * ((uint64_t)team * w + tid) + 2] = (double)sum32;
  }
  pop(s, f);
}

/* ------------------------------------------------------------------------ */
/* P4 "hetero": D levels, frame F_k = int32[L_k], L_k = S_k/4; level images */
/* are per instance (shared by its teams), level k at image_offset plus the */
/* 16-byte-padded sizes of levels < k. Level k = 1..D:                      */
/*   master: push F_k; F_k[w] = img_k[w] ^ mix32(salt + team*8 + k);         */
/*           if k > 1: F_k[0] ^= c_{k-1}.                                    */
/*   parallel, k < D: for w = tid; w < L_k; w += W': F_k[w] = mix32(F_k[w]+w) */
/*   parallel, k = D: out[team*W' + tid] =                                  */
/*           sum_{m=1..D} sum_{w = tid; w < L_m; w += W'}                    */
/*               mix32(F_m[w] ^ (m << 24) ^ w)                               */
/*   master after the join, k < D: c_k = sum_w F_k[w]; chk[k-1] = c_k.       */
/* chk[D-1] = F_D[0]. Unwind: pop F_D .. F_1.                               */
/* ------------------------------------------------------------------------ */
static void team_hetero(const orc_region *d, uint32_t team, const uint8_t *img,
                        uint8_t *out, orc_stack *s, orc_team_status *st) {
  uint32_t W = width(d), D = d->depth;
  uint8_t *F[ORC_MAX_LEVELS] = {0};
  uint32_t *o = (uint32_t *)(out + d->out_offset);
  uint64_t ioff = d->image_offset;
  uint32_t c_prev = 0;
  for (uint32_t k = 1; k <= D; k++) {
    uint32_t L = d->frame_bytes[k - 1] / 4;
    uint8_t *f = push(s, d->frame_bytes[k - 1]);
    if (!f) return;
    F[k - 1] = f;
    uint32_t key = orc_mix32(d->salt + team * 8u + k);
    for (uint32_t i = 0; i < L; i++) st32(f + 4 * i, ld32(img + ioff + 4ull * i) ^ key);
    ioff += ((uint64_t)d->frame_bytes[k - 1] + 15u) & ~(uint64_t)15u;
    if (k > 1) st32(f, ld32(f) ^ c_prev);
    for (uint32_t tid = 0; tid < W; tid++) {
      if (k < D) {
        for (uint32_t i = tid; i < L; i += W) st32(f + 4 * i, orc_mix32(ld32(f + 4 * i) + i));
      } else {
        uint32_t acc = 0;
        for (uint32_t m = 1; m <= D; m++) {
          uint32_t Lm = d->frame_bytes[m - 1] / 4;
          for (uint32_t i = tid; i < Lm; i += W)
            acc += orc_mix32(ld32(F[m - 1] + 4 * i) ^ (m << 24) ^ i);
        }
        o[(uint64_t)team * W + tid] = acc;
      }
    }
    if (k < D) {
      uint32_t c = 0;
      for (uint32_t i = 0; i < L; i++) c += ld32(f + 4 * i);
      c_prev = c;
      st->chk[k - 1] = c;
    }
  }
  st->chk[D - 1] = ld32(F[D - 1]);
  for (uint32_t k = D; k >= 1; k--) pop(s, F[k - 1]);
}

/* ------------------------------------------------------------------------ */
/* P5 "workers": sharing at worker level, the all-to-all pattern the paper  */
/* leaves to future work (Sec. 7), with each worker's frame on a stack of   */
/* its warp and the runtime-managed global stack behind it (Sec. 7); the    */
/* nested team of a worker is its warp's 32 lanes (the CUDA-NP mapping of   */
/* Sec. 2: a warp's other threads run the nested parallel region).          */
/* Image of team t at image_offset + t * (16 + pad16(S)): int32 s[4], then   */
/* int32 base[L], L = S/4, S = frame_bytes[1].                               */
/*   master: push F = s[4] (frame_bytes[0] = 16) from the image.            */
/*   outer parallel, width W': outer thread t = 0 .. W'-1:                   */
/*     push G_t = int32[L] on the stack of warp t/32;                        */
/*     G_t[i] = base[i] ^ mix32(F.s0 + t);                                   */
/*     nested parallel, 32 threads j: for w = j; w < L; w += 32:             */
/*       G_t[w] = mix32(G_t[w] + F.s1 + w);                                  */
/*     out[team*W' + t] = (sum_w G_t[w]) ^ F.s2.                             */
/*   A warp's outer threads push in lane order, all before any of their     */
/*   nested regions, and pop in reverse order.                               */
/*   master after the join: chk[0] = sum_{t < W'} out[team*W' + t]; pop F.   */
/* Warp stacks: what the team's slab and overflow slab have left after F is */
/* split evenly, in 16-byte units, over the W/32 worker warps; a warp's     */
/* stack places each frame first fit (its slab share, else its overflow     */
/* share). A push that fits neither makes the team OVERFLOW, and that outer */
/* thread runs nothing. hwm and spill add the team stack's peaks and every  */
/* warp stack's peaks.                                                      */
/* ------------------------------------------------------------------------ */
static void team_workers(const orc_region *d, uint32_t team, const uint8_t *img,
                         uint8_t *out, orc_stack *s, orc_team_status *st) {
  uint32_t Wp = width(d), L = d->frame_bytes[1] / 4;
  uint32_t nwarps = team_width(d) / 32;
  uint64_t stride = 16u + (((uint64_t)d->frame_bytes[1] + 15u) & ~(uint64_t)15u);
  const uint8_t *timg = img + d->image_offset + (uint64_t)team * stride;
  uint32_t *o = (uint32_t *)(out + d->out_offset);
  uint8_t *F = push(s, 16);
  if (!F) return;
  memcpy(F, timg, 16);
  uint64_t wslab = ((s->slab_cap - s->slab_used) / nwarps) & ~(uint64_t)15u;
  uint64_t wovf = ((s->ovf_cap - s->ovf_used) / nwarps) & ~(uint64_t)15u;
  uint64_t whwm = 0, wspill = 0;
  int failed = 0;
  for (uint32_t w = 0; w < nwarps; w++) {
    orc_stack ws;
    stack_init(&ws, wslab, wovf);
    ws.cap = ORC_WARP_CAP;
    uint8_t *G[32] = {0};
    uint32_t lanes = 0; /* outer threads of this warp */
    while (lanes < 32 && w * 32 + lanes < Wp) lanes++;
    for (uint32_t l = 0; l < lanes; l++) { /* pushes, in lane order */
      G[l] = push(&ws, d->frame_bytes[1]);
      if (!G[l]) break;
      uint32_t t = w * 32 + l, key = orc_mix32(ld32(F) + t);
      for (uint32_t i = 0; i < L; i++) st32(G[l] + 4 * i, ld32(timg + 16 + 4ull * i) ^ key);
    }
    for (uint32_t l = 0; l < lanes && G[l]; l++) { /* nested regions, then results */
      uint32_t t = w * 32 + l;
      for (uint32_t j = 0; j < 32; j++)
        for (uint32_t i = j; i < L; i += 32)
          st32(G[l] + 4 * i, orc_mix32(ld32(G[l] + 4 * i) + ld32(F + 4) + i));
      uint32_t sum = 0;
      for (uint32_t i = 0; i < L; i++) sum += ld32(G[l] + 4 * i);
      o[(uint64_t)team * Wp + t] = sum ^ ld32(F + 8);
    }
    if (ws.status != ORC_OK) failed = 1;
    whwm += ws.hwm;
    wspill += ws.spill_hwm;
    unwind(&ws); /* pops in reverse push order */
  }
  if (failed) s->status = ORC_ERR_OVERFLOW;
  s->hwm += whwm;
  s->spill_hwm += wspill;
  uint32_t c = 0;
  for (uint32_t t = 0; t < Wp; t++) c += o[(uint64_t)team * Wp + t];
  st->chk[0] = c;
  pop(s, F);
}

/* ------------------------------------------------------------------------ */
/* Descriptor checks: the sizes each program's frames must have.           */
/* ------------------------------------------------------------------------ */
static int check_region(const orc_region *d) {
  if (d->teams == 0 || d->threads < 32 || d->threads > 1024 || d->threads % 32) return 0;
  if (d->depth == 0 || d->depth > ORC_MAX_LEVELS) return 0;
  if (d->width > team_width(d)) return 0;
  for (uint32_t k = 0; k < d->depth; k++)
    if (d->frame_bytes[k] == 0 || d->frame_bytes[k] % 4) return 0;
  uint32_t w = width(d);
  switch (d->program) {
    case PROG_PAPER_SCALARS:
      return d->depth == 1 && d->param >= 1 &&
             d->frame_bytes[0] == ((4u * d->param + 7u) & ~7u) + 8u;
    case PROG_PAPER_ARRAYS:
      return d->depth == 1 && d->param >= 1 && d->frame_bytes[0] == 4u * d->param * w;
    case PROG_SCALARS:
      return d->depth == 1 && d->frame_bytes[0] == 16 && d->param >= 1;
    case PROG_NESTED:
      for (uint32_t k = 0; k < d->depth; k++)
        if (d->frame_bytes[k] != 1088) return 0;
      return d->param >= 1;
    case PROG_SWEEP:
      return d->depth == 1;
    case PROG_HETERO:
      return 1;
    case PROG_WORKERS:
      return d->depth == 2 && d->frame_bytes[0] == 16 && d->threads >= 64;
    default:
      return 0;
  }
}

/*
 * Run teams [team_begin, team_end) of one region instance.
 *   images: the image buffer (the descriptor's image_offset indexes it).
 *   out:    the output buffer (out_offset indexes it). For the sweep
 *           program it holds double[T][W'][3] (fp64 sum, fp64 sum of
 *           magnitudes, fp32 sum), at 6 * out_offset bytes.
 *   status: the team-status array; team t writes status[status_index + t].
 *   slab_bytes / overflow_bytes: stack capacities per team.
 * Returns ORC_OK, or ORC_ERR_INVALID for a malformed descriptor.
 */
int orc_run(const orc_region *d, const uint8_t *images, uint8_t *out, orc_team_status *status,
            uint64_t slab_bytes, uint64_t overflow_bytes, uint32_t team_begin,
            uint32_t team_end) {
  if (!check_region(d)) return ORC_ERR_INVALID;
  if (team_end > d->teams) team_end = d->teams;
  for (uint32_t team = team_begin; team < team_end; team++) {
    orc_stack s;
    orc_team_status st;
    memset(&st, 0, sizeof(st));
    stack_init(&s, slab_bytes, overflow_bytes);
    switch (d->program) {
      case PROG_PAPER_SCALARS: team_paper_scalars(d, team, out, &s); break;
      case PROG_PAPER_ARRAYS: team_paper_arrays(d, team, out, &s); break;
      case PROG_SCALARS: team_scalars(d, team, images, out, &s); break;
      case PROG_NESTED: team_nested(d, team, images, out, &s, &st); break;
      case PROG_SWEEP: team_sweep(d, team, images, out, &s); break;
      case PROG_HETERO: team_hetero(d, team, images, out, &s, &st); break;
      case PROG_WORKERS: team_workers(d, team, images, out, &s, &st); break;
    }
    if (s.status != ORC_OK) memset(st.chk, 0, sizeof(st.chk));
    unwind(&s); /* no-op for a program that popped everything */
    st.status = s.status;
    st.depth_final = s.depth;
    st.hwm_bytes = (uint32_t)s.hwm;
    st.spill_bytes = (uint32_t)s.spill_hwm;
    status[d->status_index + team] = st;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Stack primitives exported for the allocator tests (LIFO misuse and       */
/* capacity cases are exercised here, on the CPU).                          */
/* ------------------------------------------------------------------------ */
void *orc_stack_new(uint64_t slab_bytes, uint64_t overflow_bytes) {
  orc_stack *s = (orc_stack *)malloc(sizeof(orc_stack));
  if (s) stack_init(s, slab_bytes, overflow_bytes);
  return s;
}
void orc_stack_free(void *h) {
  orc_stack *s = (orc_stack *)h;
  if (!s) return;
  unwind(s);
  free(s);
}
/* Returns the frame's index in the table, or -1 when the push fails. */
int orc_stack_push(void *h, uint32_t bytes, int *in_slab) {
  orc_stack *s = (orc_stack *)h;
  if (!push(s, bytes)) return -1;
  if (in_slab) *in_slab = s->f[s->depth - 1].in_slab;
  return (int)s->depth - 1;
}
/* Pops the frame at table index `idx`; LIFO misuse returns ORC_ERR_LIFO. */
int orc_stack_pop(void *h, int idx) {
  orc_stack *s = (orc_stack *)h;
  if (idx < 0 || (uint32_t)idx >= s->depth) {
    s->status = ORC_ERR_LIFO;
    return ORC_ERR_LIFO;
  }
  return pop(s, s->f[idx].data);
}
void orc_stack_state(void *h, uint64_t out[6]) {
  orc_stack *s = (orc_stack *)h;
  out[0] = s->depth;
  out[1] = s->slab_used;
  out[2] = s->ovf_used;
  out[3] = s->hwm;
  out[4] = s->spill_hwm;
  out[5] = (uint64_t)(int64_t)s->status;
}
