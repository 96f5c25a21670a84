// user_programs.cu -- two region programs written outside the library,
// against the public device API of dsr_device.cuh only, to show that a
// user's own program runs through the runtime's plain and batched launches.
// Test infrastructure: the GPU tests load the shared library built from
// this file and compare its results with the CPU oracle's programs of the
// same definition.
//
//  * UserPaperScalars (Sec. 6.1, Fig. "Implicitly sharing 8 variables"):
//    the sequential code declares int c_1..c_n and the reference to the
//    mapped array a, sets every c_i to 0 and then adds i to c_i; the nested
//    parallel region adds the sum of the c_i to a[team*W' + tid]. The frame
//    holds the n ints and, 8-byte aligned after them, the reference.
//  * UserHetero: the heterogeneous-instance program. Level k = 1..D pushes
//    F_k = int32[L_k] filled from the instance's level image and keyed with
//    mix32(salt + team*8 + k), F_k[0] ^= c_{k-1} for k > 1; region k < D
//    updates F_k[w] = mix32(F_k[w] + w) and the master then sums F_k into
//    c_k (check word k-1); the innermost region writes
//    out[team*W' + tid] = sum over m <= D and w = tid, tid + W', ... of
//    mix32(F_m[w] ^ (m << 24) ^ w); check word D-1 = F_D[0]; the frames
//    are popped D .. 1.
#include <cstdint>

#include "dsr_device.cuh"

namespace {

// 32-bit finaliser of MurmurHash3 (Appleby, public domain): the programs'
// own hash.
__host__ __device__ __forceinline__ uint32_t user_mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__host__ __device__ __forceinline__ uint64_t user_pad16(uint64_t n) { return (n + 15u) & ~15ull; }

__host__ __device__ __forceinline__ uint32_t user_width(const dsr_region_desc &d) {
  const uint32_t w = d.threads > 32u ? d.threads - 32u : 1u;
  return d.width ? d.width : w;
}

struct UserPaperScalars {
  static constexpr uint32_t kProgram = DSR_PROG_USER + 1;

  __host__ __device__ static uint32_t ref_offset(uint32_t n) { return (4u * n + 7u) & ~7u; }

  __host__ __device__ static void extent(const dsr_region_desc &d, uint64_t *image_bytes,
                                         uint64_t *out_bytes) {
    *image_bytes = 0;
    *out_bytes = 4ull * d.teams * user_width(d);
  }

  __device__ static void master(dsr_team &t) {
    const dsr_region_desc &d = dsr_desc(t);
    const uint32_t n = d.param;
    if (d.frame_bytes[0] < ref_offset(n) + 8u) {
      // a frame too small for its variables: push nothing, run nothing
      return;
    }
    uint8_t *f = static_cast<uint8_t *>(dsr_push(t, d.frame_bytes[0]));
    if (!f) return;
    if (dsr_is_master()) {  // the sequential code, as written, by the master alone
      int32_t *c = reinterpret_cast<int32_t *>(f);
      for (uint32_t i = 0; i < n; ++i) c[i] = 0;
      for (uint32_t i = 0; i < n; ++i) c[i] += static_cast<int32_t>(i + 1);
      *reinterpret_cast<int32_t **>(f + ref_offset(n)) =
          reinterpret_cast<int32_t *>(dsr_out(t) + d.out_offset);
    }
    dsr_master_sync();
    dsr_parallel(t, 0, dsr_region_width(t), n);
    dsr_pop(t, f);
  }

  __device__ static void body(const dsr_thread &w) {
    const uint32_t n = dsr_arg(w);
    const uint8_t *f = static_cast<const uint8_t *>(dsr_frame(0));
    const int32_t *c = reinterpret_cast<const int32_t *>(f);
    int32_t *a = *reinterpret_cast<int32_t *const *>(f + ref_offset(n));
    uint32_t sum = 0;
    for (uint32_t i = 0; i < n; ++i) sum += static_cast<uint32_t>(c[i]);
    uint32_t *slot = reinterpret_cast<uint32_t *>(
        a + static_cast<uint64_t>(dsr_team_num(w)) * dsr_num_threads(w) + dsr_thread_num(w));
    *slot += sum;
  }
};

struct UserHetero {
  static constexpr uint32_t kProgram = DSR_PROG_USER + 6;
  enum : uint32_t { kUpdate = 0, kInner = 1 };

  __host__ __device__ static void extent(const dsr_region_desc &d, uint64_t *image_bytes,
                                         uint64_t *out_bytes) {
    uint64_t ib = 0;
    for (uint32_t k = 0; k < d.depth && k < DSR_MAX_DEPTH; ++k) ib += user_pad16(d.frame_bytes[k]);
    *image_bytes = ib;
    *out_bytes = 4ull * d.teams * user_width(d);
  }

  // the instance's images towards L2 before the launch waits (team 0 asks
  // for them; every team reads the same ones)
  __device__ static void prefetch(const dsr_region_desc &d, const uint8_t *images, uint32_t team) {
    uint64_t ib, ob;
    extent(d, &ib, &ob);
    if (team == 0) dsr_prefetch_l2(images + d.image_offset, static_cast<uint32_t>(ib));
  }

  __device__ static void master(dsr_team &t) {
    const dsr_region_desc &d = dsr_desc(t);
    const uint32_t D = d.depth, team = dsr_team_num(t), lane = dsr_lane();
    const uint8_t *img = dsr_images(t) + d.image_offset;
    uint32_t c_prev = 0;
    for (uint32_t k = 1; k <= D; ++k) {
      const uint32_t S = d.frame_bytes[k - 1], L = S / 4u;
      uint32_t *f = static_cast<uint32_t *>(dsr_push(t, S));
      if (!f) return;
      dsr_fill(t, f, img, S);
      if (dsr_get_status(t) != DSR_OK) return;
      // keying the words is order-free: the master warp's lanes split it
      const uint32_t key = user_mix32(d.salt + team * 8u + k);
      for (uint32_t w = lane; w < L; w += 32u) f[w] ^= key;
      dsr_master_sync();
      if (k > 1 && dsr_is_master()) f[0] ^= c_prev;
      dsr_master_sync();
      img += user_pad16(S);
      dsr_parallel(t, k < D ? kUpdate : kInner, dsr_region_width(t), k);
      if (k < D) {
        // c_k = sum of F_k (wrap-around, so the lanes' split sums agree)
        uint32_t part = 0;
        for (uint32_t w = lane; w < L; w += 32u) part += f[w];
        c_prev = __reduce_add_sync(0xffffffffu, part);
        dsr_set_check(t, k - 1, c_prev);
      }
    }
    dsr_master_sync();
    dsr_set_check(t, D - 1, static_cast<const uint32_t *>(dsr_frame(D - 1))[0]);
    for (uint32_t k = D; k >= 1; --k) dsr_pop(t, dsr_frame(k - 1));
  }

  __device__ static void body(const dsr_thread &w) {
    const uint32_t k = dsr_arg(w), tid = dsr_thread_num(w), n = dsr_num_threads(w);
    if (dsr_body(w) == kUpdate) {
      uint32_t *f = static_cast<uint32_t *>(dsr_frame(k - 1));
      const uint32_t L = dsr_frame_bytes(k - 1) / 4u;
      for (uint32_t i = tid; i < L; i += n) f[i] = user_mix32(f[i] + i);
      return;
    }
    uint32_t acc = 0;
    for (uint32_t m = 1; m <= k; ++m) {
      const uint32_t *f = static_cast<const uint32_t *>(dsr_frame(m - 1));
      const uint32_t L = dsr_frame_bytes(m - 1) / 4u;
      for (uint32_t i = tid; i < L; i += n) acc += user_mix32(f[i] ^ (m << 24) ^ i);
    }
    const dsr_region_desc &d = dsr_desc(w);
    reinterpret_cast<uint32_t *>(dsr_out(w) + d.out_offset)
        [static_cast<uint64_t>(dsr_team_num(w)) * n + tid] = acc;
  }
};

}  // namespace

// The plain kernel finds the optional prefetch through the adapter.
static_assert(dsr::has_prefetch<dsr::UserProgram<UserHetero>>::value, "prefetch hook");
static_assert(!dsr::has_prefetch<dsr::UserProgram<UserPaperScalars>>::value, "no prefetch hook");

// ---- C entry points the tests call (ctypes) -------------------------------
#define USER_ENTRY(name, Prog)                                                                 \
  extern "C" int32_t name##_launch(dsr_ctx *ctx, const dsr_region_desc *d, const void *images, \
                                   uint64_t image_bytes, void *out, uint64_t out_bytes,        \
                                   dsr_team_status *status, uint64_t n_status, void *stream) { \
    return dsr_launch_user_region<Prog>(ctx, d, images, image_bytes, out, out_bytes, status,   \
                                        n_status, stream);                                     \
  }                                                                                            \
  extern "C" int32_t name##_launch_batch(                                                      \
      dsr_ctx *ctx, const dsr_region_desc *descs, uint32_t n, uint64_t total_teams,            \
      const void *images, uint64_t image_bytes, void *out, uint64_t out_bytes,                 \
      dsr_team_status *status, uint64_t n_status, void *ws, uint64_t ws_bytes,                 \
      const dsr_batch_tuning *tuning, void *stream) {                                          \
    return dsr_launch_user_batch<Prog>(ctx, descs, n, total_teams, images, image_bytes, out,   \
                                       out_bytes, status, n_status, ws, ws_bytes, tuning,      \
                                       stream);                                                \
  }                                                                                            \
  extern "C" int32_t name##_serve_start(dsr_ctx *ctx, const dsr_serve_cfg *cfg, void *ws,      \
                                        uint64_t ws_bytes) {                                   \
    return dsr_serve_user_start<Prog>(ctx, cfg, ws, ws_bytes);                                 \
  }                                                                                            \
  extern "C" const dsr_serve_program *name##_serve_program(void) {                             \
    return dsr_serve_user_program<Prog>();                                                     \
  }                                                                                            \
  extern "C" uint32_t name##_program(void) { return Prog::kProgram; }

USER_ENTRY(user_paper_scalars, UserPaperScalars)
USER_ENTRY(user_hetero, UserHetero)
