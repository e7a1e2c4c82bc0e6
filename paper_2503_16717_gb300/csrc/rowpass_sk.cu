// The sketch row pass with its two kinds of work on separate warps.
//
// A pass that applies the sparse sketch (BCGS update + RandHH sketch of the one-stage
// scheme, Section 5; update + sketched BCGS2-HH of the two-stage scheme, Section 7;
// the standalone sketch apply) does per row tile
//   (U) y' = (y - x C) [Tri^-1] and its write-back: float64 FMAs, bound by the
//       float64 pipe;
//   (S) S y': the exponent maximum of each column, the values as int64 fixed point
//       and the exact integer sums of the tile's entries per sketch row: integer
//       issue and shared-memory bound.
// In one CTA the first 4 warps (one per SM sub-partition) run U on tile i + 1 while
// the other 4 run S on tile i.  The X columns of a tile sit in a ring of 2 stages
// (only U reads them), its Y columns and schedule record in a ring of 3; mbarriers
// hand a Y stage from the copy engine to U (full), from U to S (ready) and from S back
// to the copy engine (free).  Every wait is bounded; a wait that gives up raises a
// CTA-wide abort flag that ends the other group's waits too.
//
// The sums are those of the single-group kernel: each sketch row of a tile is summed
// by one thread in increasing tile row (exactly, in integers), and the tile sums enter
// the float64 accumulators in the CTA's tile order.
#include <algorithm>
#include <mutex>

#include "rowpass_common.cuh"

namespace rbo {

constexpr int SK_UW = 4;                 // transform warps (U)
constexpr int SK_SW = 4;                 // sketch warps (S)
constexpr int SK_NT = 32 * (SK_UW + SK_SW);
constexpr int SK_MINB = SK_NT <= 256 ? 4 : 3;  // CTAs per SM the registers allow
constexpr int SK_UN = SK_UW * 32;
constexpr int SK_SN = SK_SW * 32;
constexpr int SK_XST = 2;                // X stages
constexpr int SK_YST = 3;                // Y stages
constexpr int SK_BAR_BYTES = 128;        // 3 x 3 mbarriers at the start of shared memory

__device__ __forceinline__ void mbar_arrive_plain(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}
// barrier among the `count` threads of one warp group (ids 1 and 2; 0 is __syncthreads)
__device__ __forceinline__ void group_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// y' = y Tri^-1 in place over the tile's rows, by the U group: column blocks of CB;
// the block's update by the finished columns over all (row, column) pairs, the
// substitution inside the block by rows, every entry subtracting its terms in column
// order (as an unblocked row-by-row substitution would).
__device__ __forceinline__ void sk_tri_solve(double* ys, const double* Ts, const double* dinv, int T,
                                             int TP, int b, int ut, bool dead) {
  for (int c0 = 0; c0 < b; c0 += CB) {
    const int cw = min(CB, b - c0);
    if (c0 > 0) {
      if (!dead) {
        for (int t = ut; t < T * cw; t += SK_UN) {
          const int r = t % T, c = c0 + t / T;
          double v = ys[c * TP + r];
          for (int i = 0; i < c0; ++i) v = fma(-ys[i * TP + r], Ts[i + c * b], v);
          ys[c * TP + r] = v;
        }
      }
      group_bar(1, SK_UN);
    }
    if (!dead) {
      for (int r = ut; r < T; r += SK_UN) {
        for (int c = c0; c < c0 + cw; ++c) {
          double v = ys[c * TP + r];
          for (int i = c0; i < c; ++i) v = fma(-ys[i * TP + r], Ts[i + c * b], v);
          ys[c * TP + r] = v * dinv[c];
        }
      }
    }
    if (c0 + CB < b) group_bar(1, SK_UN);
  }
}
// y' = y - x C in place, one (row, column) element per task, two interleaved chains
__device__ __forceinline__ void sk_project(double* ys, const double* xs, const double* Cs, int T,
                                           int TP, int a, int b, int ut) {
  for (int t = ut; t < T * b; t += SK_UN) {
    const int r = t % T, c = t / T;
    const double* cc = Cs + (size_t)c * a;
    double v0 = ys[c * TP + r], v1 = 0.0;
    int i = 0;
    for (; i + 1 < a; i += 2) {
      v0 = fma(-xs[i * TP + r], cc[i], v0);
      v1 = fma(-xs[(i + 1) * TP + r], cc[i + 1], v1);
    }
    if (i < a) v0 = fma(-xs[i * TP + r], cc[i], v0);
    ys[c * TP + r] = v0 + v1;
  }
}

template <int ARITH>
__global__ void __launch_bounds__(SK_NT, SK_MINB) rowpass_sk_kernel(const __grid_constant__ PassDev P) {
  // ARITH 0: float64 transform, exact fixed-point sketch sums; 1 (mixed precision):
  // float64 transform, float32 sketch sums.
  constexpr bool MIXED = ARITH == 1;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ int s_last;
  __shared__ int s_abort;
  __shared__ int s_pend[SK_YST];          // copy in flight into Y stage y: its parity + 1
  __shared__ int s_emax[SK_YST][64];      // per Y stage: largest exponent field per column
  const RowPass& rp = P.p;
  if (read_code(P.status) != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = P.T, TP = P.TP, a = rp.a, b = rp.b, d = rp.sk_d;
  const int64_t n = rp.n;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* ready = full + SK_YST;
  uint64_t* freeb = ready + SK_YST;
  double* Cs = reinterpret_cast<double*>(smem + P.off_c);
  double* Ts = reinterpret_cast<double*>(smem + P.off_tri);
  double* dinv = reinterpret_cast<double*>(smem + P.off_dinv);
  double* skd = reinterpret_cast<double*>(smem + P.off_sk);
  float* skf = reinterpret_cast<float*>(smem + P.off_sk);

  if (rp.C) {
    const int ldc = rp.ldc > 0 ? rp.ldc : a;
    for (int t = tid; t < a * b; t += SK_NT) Cs[t] = rp.C[(t % a) + (size_t)(t / a) * ldc];
  }
  if (rp.Tri) {
    const int ldt = rp.ldtri > 0 ? rp.ldtri : b;
    for (int t = tid; t < b * b; t += SK_NT) {
      const int i = t % b, c = t / b;
      Ts[t] = (i <= c) ? rp.Tri[i + (size_t)c * ldt] : 0.0;
    }
    for (int t = tid; t < b; t += SK_NT) dinv[t] = 1.0 / rp.Tri[t + (size_t)t * ldt];
  }
  for (int t = tid; t < d * b; t += SK_NT) {
    if (MIXED)
      skf[t] = 0.0f;
    else
      skd[t] = 0.0;
  }
  if (tid == 0) {
    for (int y = 0; y < SK_YST; ++y) {
      mbar_init(&full[y], 1);
      mbar_init(&ready[y], SK_UN);
      mbar_init(&freeb[y], SK_SN);
      s_pend[y] = 0;
    }
    s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();

  const int rec_n = rp.sk.rec_bytes;
  auto stage_X = [&](int it) {
    return reinterpret_cast<double*>(smem + P.off_stage + (size_t)(it & 1) * P.stage_bytes);
  };
  auto stage_Y = [&](int it) {
    return reinterpret_cast<double*>(smem + P.off_ys + (size_t)(it % SK_YST) * P.ystage_bytes);
  };
  auto stage_R = [&](int it) {
    return smem + P.off_ys + (size_t)(it % SK_YST) * P.ystage_bytes + P.rec_off;
  };
  auto bulk_ok = [&](int tile) { return P.use_bulk && ((int64_t)(tile + 1) * T <= n); };
  // Bounded wait that also ends once any thread gave up (s_abort).  A thread that
  // failed a wait is `dead`: it skips the work and the copies but still passes every
  // group barrier of its loop, so the groups never wait on a thread that left.
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
      if (mbar_try_wait(bar, parity)) return true;
      if (*reinterpret_cast<volatile int*>(&s_abort)) return false;
      if (clock64() - t0 > WAIT_CYCLES) {
        atomicExch(&s_abort, 1);
        return false;
      }
    }
  };
  // copy tile `tile` (the CTA's it-th) into X stage it & 1 and Y stage it % 3 (warp 0)
  auto issue_tile = [&](int tile, int it) {
    const int64_t r0 = (int64_t)tile * T;
    double* xs = stage_X(it);
    double* ys = stage_Y(it);
    uint64_t* bar = &full[it % SK_YST];
    const uint32_t bytes = (uint32_t)T * 8u;
    if (lane == 0) {
      s_pend[it % SK_YST] = (int)((it / SK_YST) & 1) + 1;
      mbar_arrive_expect_tx(bar, bytes * (uint32_t)(a + b) + (uint32_t)rec_n);
    }
    __syncwarp();
    for (int j = lane; j < a + b + 1; j += 32) {
      if (j < a)
        bulk_copy_g2s(xs + (size_t)j * TP, rp.X + j * rp.ldx + r0, bytes, bar);
      else if (j < a + b)
        bulk_copy_g2s(ys + (size_t)(j - a) * TP, rp.Y + (j - a) * rp.ldy + r0, bytes, bar);
      else
        bulk_copy_g2s(stage_R(it), rp.sk.rec + (size_t)tile * rec_n, (uint32_t)rec_n, bar);
    }
  };
  const int first = blockIdx.x;
  bool dead = false;

  if (warp < SK_UW) {
    // ---------------- U: transform + write-back ----------------------------------
    const int ut = tid;
    if (warp == 0 && first < P.ntiles && bulk_ok(first)) issue_tile(first, 0);
    int it = 0;
    for (int tile = first; tile < P.ntiles; tile += gridDim.x, ++it) {
      const int64_t r0 = (int64_t)tile * T;
      const int rows = (n - r0 < (int64_t)T) ? (int)(n - r0) : T;
      const uint32_t par = (uint32_t)((it / SK_YST) & 1);
      double* xs = stage_X(it);
      double* ys = stage_Y(it);
      if (bulk_ok(tile)) {
        if (!dead && !wait(&full[it % SK_YST], par)) dead = true;
        if (ut == 0 && !dead) s_pend[it % SK_YST] = 0;
      } else {
        // ragged or unaligned tile: plain loads with zero fill, once S has released
        // the Y stage (its use three tiles back)
        if (!dead && it >= SK_YST && !wait(&freeb[it % SK_YST], par ^ 1u)) dead = true;
        if (!dead) {
          for (int t = ut; t < a * T; t += SK_UN) {
            const int col = t / T, r = t % T;
            xs[(size_t)col * TP + r] = r < rows ? rp.X[col * rp.ldx + r0 + r] : 0.0;
          }
          for (int t = ut; t < b * T; t += SK_UN) {
            const int col = t / T, r = t % T;
            ys[(size_t)col * TP + r] = r < rows ? rp.Y[col * rp.ldy + r0 + r] : 0.0;
          }
          uint32_t* es = reinterpret_cast<uint32_t*>(stage_R(it));
          const uint32_t* eg = reinterpret_cast<const uint32_t*>(rp.sk.rec + (size_t)tile * rec_n);
          for (int t = ut; t < rec_n / 4; t += SK_UN) es[t] = eg[t];
        }
        group_bar(1, SK_UN);
      }
      // prefetch the next tile into the stages of it + 1 once S has released that Y
      // stage (lane 0 waits for the warp; the copies need the whole warp)
      const int nxt = tile + gridDim.x;
      if (warp == 0 && nxt < P.ntiles && bulk_ok(nxt)) {
        const int it1 = it + 1;
        bool ok = !dead;
        if (ok && lane == 0 && it1 >= SK_YST)
          ok = wait(&freeb[it1 % SK_YST], (uint32_t)(((it1 / SK_YST) & 1) ^ 1));
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) {
          fence_proxy_async();
          issue_tile(nxt, it1);
        } else {
          dead = true;
        }
      }
      // y' = (y - x C) Tri^-1 (or y Tri^-1 - x C) in place in the Y stage
      if (rp.Tri && rp.tri_first) {
        sk_tri_solve(ys, Ts, dinv, T, TP, b, ut, dead);
        group_bar(1, SK_UN);
      }
      if (rp.C) {
        if (!dead) sk_project(ys, xs, Cs, T, TP, a, b, ut);
        group_bar(1, SK_UN);
      }
      if (rp.Tri && !rp.tri_first) {
        sk_tri_solve(ys, Ts, dinv, T, TP, b, ut, dead);
        group_bar(1, SK_UN);
      }
      if (rp.write_y && !dead) {
        for (int t = ut; t < b * T; t += SK_UN) {
          const int c = t / T, rr = t % T;
          if (rr < rows) rp.Y[c * rp.ldy + r0 + rr] = ys[(size_t)c * TP + rr];
        }
      }
      if (!dead) mbar_arrive_plain(&ready[it % SK_YST]);
      // every U thread is done with X stage it & 1 before warp 0 copies into it again
      group_bar(1, SK_UN);
    }
  } else {
    // ---------------- S: exponent maxima, fixed point, entry sums -----------------
    const int stid = tid - SK_UN, sw = warp - SK_UW;
    int it = 0;
    for (int tile = first; tile < P.ntiles; tile += gridDim.x, ++it) {
      const int64_t r0 = (int64_t)tile * T;
      const int rows = (n - r0 < (int64_t)T) ? (int)(n - r0) : T;
      const int y = it % SK_YST;
      if (!dead && !wait(&ready[y], (uint32_t)((it / SK_YST) & 1))) dead = true;
      dead = __any_sync(0xffffffffu, dead);
      double* ys = stage_Y(it);
      if (!MIXED) {
        // per column: the largest exponent field of the tile (one warp per column),
        // then the values in place as int64 fixed point
        if (!dead) {
          for (int c = sw; c < b; c += SK_SW) {
            int ex = 0;
            for (int r = lane; r < T; r += 32) {
              const unsigned long long u =
                  (unsigned long long)__double_as_longlong(ys[(size_t)c * TP + r]);
              if (r < rows) ex = max(ex, (int)((u >> 52) & 0x7FF));
            }
            ex = __reduce_max_sync(0xffffffffu, ex);
            if (lane == 0) s_emax[y][c] = ex;
          }
        }
        group_bar(2, SK_SN);
        if (!dead) {
          for (int t = stid; t < b * T; t += SK_SN) {
            const int c = t / T, r = t % T;
            const int E = s_emax[y][c];
            const double yv = ys[(size_t)c * TP + r];
            reinterpret_cast<long long*>(ys)[(size_t)c * TP + r] =
                (r < rows && E != 0x7FF) ? fix_from_double(yv, E) : 0LL;
          }
        }
      } else {
        // float32 copies in place: the float of element t in the first 4 bytes of its slot
        if (!dead) {
          for (int t = stid; t < b * T; t += SK_SN) {
            const size_t e = (size_t)(t / T) * TP + (t % T);
            const float f = f64_to_f32_int(ys[e]);
            reinterpret_cast<float*>(ys + e)[0] = f;
          }
        }
      }
      group_bar(2, SK_SN);
      // the record lists the tile's non-empty sketch rows, most entries first; thread
      // q adds the entries of the rows in slots q, q + 128, ... (no other thread
      // touches those accumulators during the tile)
      if (!dead) {
        const uint32_t* meta = reinterpret_cast<const uint32_t*>(stage_R(it));
        const uint8_t* lst = reinterpret_cast<const uint8_t*>(meta + rp.sk.mcap);
        for (int q = stid; q < rp.sk.mcap; q += SK_SN) {
          const uint32_t m = meta[q];
          if (m == 0xFFFFFFFFu) break;
          const int i = (int)(m & 0xFFFu), o = (int)((m >> 12) & 0x7FFu), cnt = (int)(m >> 23);
          const uint8_t* e = lst + o;
          for (int c0 = 0; c0 < b; c0 += CB) {
            const int cw = min(CB, b - c0);
            if (MIXED) {
              RBO_CW_DISPATCH(sketch_row_f32, cw, skf + i + (size_t)c0 * d, d,
                              reinterpret_cast<const float*>(ys + (size_t)c0 * TP), 2 * TP, e, cnt)
            } else {
              RBO_CW_DISPATCH(sketch_row_fix, cw, skd + i + (size_t)c0 * d, d,
                              reinterpret_cast<const long long*>(ys) + (size_t)c0 * TP, TP,
                              s_emax[y] + c0, e, cnt)
            }
          }
        }
        mbar_arrive_plain(&freeb[y]);
      }
    }
  }
  __syncthreads();
  if (s_abort) {
    // the copies still in flight land before the CTA leaves
    if (tid == 0) {
      set_error(P.status, RBO_ERR_TIMEOUT, 1);
      for (int y = 0; y < SK_YST; ++y)
        if (s_pend[y]) mbar_wait_bounded(&full[y], (uint32_t)(s_pend[y] - 1));
    }
    return;
  }

  // ---------------- partial + fixed-order two-level tree -------------------------
  double* mypart = P.partials + (size_t)blockIdx.x * P.L;
  for (int t = tid; t < d * b; t += SK_NT) mypart[t] = MIXED ? (double)skf[t] : skd[t];
  tree_reduce_epilogue(P, smem, &s_flag, &s_last);
}

// ------------------------------------------------------------------------------------
// launcher
// ------------------------------------------------------------------------------------
constexpr int SK_MAX_DEV = 64;
static std::mutex g_sk_mu;
static int g_sk_smem[SK_MAX_DEV][2] = {};

// Shared-memory bytes of the streaming loop: mbarriers, 2 X stages, 3 Y stages (Y
// columns + schedule record), C, Tri, 1/diag, the sketch accumulators.
struct SkLayout {
  size_t off_stage, xstage, off_ys, ystage, rec_off, off_c, off_tri, off_dinv, off_sk, loop_bytes;
};
static SkLayout sk_layout(int a, int b, int T, int rec_bytes, int d, bool has_c, bool has_tri,
                          bool mixed) {
  SkLayout l;
  const size_t TP = (size_t)T + 2;
  l.off_stage = SK_BAR_BYTES;
  l.xstage = (size_t)a * TP * 8;  // TP even: a 16-byte multiple
  l.off_ys = l.off_stage + SK_XST * l.xstage;
  l.rec_off = (size_t)b * TP * 8;
  l.ystage = l.rec_off + (size_t)rec_bytes;
  size_t o = l.off_ys + SK_YST * l.ystage;
  l.off_c = o; o += has_c ? (size_t)a * b * 8 : 0;
  l.off_tri = o; o += has_tri ? (size_t)b * b * 8 : 0;
  l.off_dinv = o; o += has_tri ? (size_t)b * 8 : 0;
  o = (o + 15) & ~size_t(15);
  l.off_sk = o; o += (size_t)d * b * (mixed ? 4 : 8);
  l.loop_bytes = (o + 15) & ~size_t(15);
  return l;
}

size_t rowpass_sk_loop_bytes(int a, int b, int T, int d, int zeta) {
  return sk_layout(a, b, T, sketch_sched_rec_bytes(T, d, zeta), d, a > 0, true, false).loop_bytes;
}

template <int ARITH>
static int sk_smem_limit(int dev) {
  std::lock_guard<std::mutex> lk(g_sk_mu);
  int& lim = g_sk_smem[dev][ARITH];
  if (lim == 0) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    size_t stat = 0;
    if (cudaFuncGetAttributes(&fa, rowpass_sk_kernel<ARITH>) == cudaSuccess) stat = fa.sharedSizeBytes;
    lim = optin - (int)stat - 64;
    if (cudaFuncSetAttribute(rowpass_sk_kernel<ARITH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             lim) != cudaSuccess) {
      cudaGetLastError();
      lim = 48 * 1024 - (int)stat;
    }
  }
  return lim;
}

template <int ARITH>
static int sk_occupancy(int smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rowpass_sk_kernel<ARITH>, SK_NT, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  return nb < 1 ? 1 : nb;
}

int rowpass_sk_launch(const RowPass& rp, Arena* ar, cudaStream_t st, int* launches, int num_sms,
                      int L, int mixed) {
  const int d = rp.sk_d, T = rp.sk.T;
  if (d <= 0 || T < 16 || T > 128 || (T & 15) != 0) return RBO_ERR_ARG;
  if (rp.b > 64) return RBO_ERR_ARG;  // s_emax holds 64 columns
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SK_MAX_DEV) dev = 0;
  const SkLayout l = sk_layout(rp.a, rp.b, T, rp.sk.rec_bytes, d, rp.C != nullptr,
                               rp.Tri != nullptr, mixed != 0);
  const size_t off_red = SK_BAR_BYTES;
  const size_t epi_bytes = off_red + ((size_t)L + 2) * 8 + epilogue_doubles(rp) * 8;
  const size_t smem = std::max(l.loop_bytes, epi_bytes);
  const int limit = mixed ? sk_smem_limit<1>(dev) : sk_smem_limit<0>(dev);
  if ((long long)smem > limit) return RBO_ERR_ARG;
  const int ntiles = (int)((rp.n + T - 1) / T);
  const int occ = mixed ? sk_occupancy<1>((int)smem) : sk_occupancy<0>((int)smem);
  int G = std::min(ntiles, occ * num_sms);
  if (rp.max_ctas > 0) G = std::min(G, rp.max_ctas);
  if (G < 1) G = 1;
  const int ngroups = (G + GROUP - 1) / GROUP;

  PassDev P;
  P.p = rp;
  P.T = T;
  P.TP = T + 2;
  P.ntiles = ntiles;
  P.items = 0;
  P.cw = 1;
  P.nblk = 0;
  for (int k = 0; k < 9; ++k) P.blk_start[k] = 0;
  P.tpo = 1;
  P.tasks = 0;
  P.flush_tiles = 1;
  const bool alignedX = rp.a == 0 || (((uintptr_t)rp.X & 15) == 0 && (rp.ldx % 2) == 0);
  const bool alignedY = (((uintptr_t)rp.Y & 15) == 0 && (rp.ldy % 2) == 0);
  P.use_bulk = (alignedX && alignedY) ? 1 : 0;
  P.zr = 0;
  P.no = 0;
  P.L = L;
  P.ngroups = ngroups;
  P.status = ar->status;
  P.off_stage = (int)l.off_stage;
  P.stage_bytes = (int)l.xstage;
  P.off_ys = (int)l.off_ys;
  P.ystage_bytes = (int)l.ystage;
  P.rec_off = (int)l.rec_off;
  P.off_c = (int)l.off_c;
  P.off_tri = (int)l.off_tri;
  P.off_dinv = (int)l.off_dinv;
  P.off_sk = (int)l.off_sk;
  P.off_gth = 0;
  P.off_red = (int)off_red;
  // reduction scratch reserved for the whole call (stream-ordered reuse); the tickets
  // were zeroed at the start of the call and every tree resets its own
  const size_t need = ((size_t)G * L + (size_t)ngroups * L) * 8;
  if (ar->red == nullptr || need > ar->red_bytes) return RBO_ERR_NOMEM;
  if (ngroups + 1 > ar->n_tickets) return RBO_ERR_NOMEM;
  P.partials = ar->red;
  P.gpart = ar->red + (size_t)G * L;
  P.tickets = ar->tickets;

  ProfToken tok = prof_start(st);
  if (mixed)
    rowpass_sk_kernel<1><<<G, SK_NT, smem, st>>>(P);
  else
    rowpass_sk_kernel<0><<<G, SK_NT, smem, st>>>(P);
  if (prof_on()) {
    // algorithmic traffic: every n-row column read once, written once
    const double nn = (double)rp.n, A = rp.a, B = rp.b;
    const bool readx = rp.a > 0 && rp.C;
    const double by = 8.0 * nn * ((readx ? A : 0.0) + B + (rp.write_y ? B : 0.0));
    double fl = 0.0;
    if (rp.C) fl += 2.0 * nn * A * B;                   // projection
    if (rp.Tri) fl += nn * B * B;                        // triangular solve
    fl += nn * (double)rp.sk_zeta * B;                   // sketch accumulation
    prof_stop(tok, st, 0, by, fl, rp.tag);
  }
  if (launches) ++*launches;
  return note_cuda(cudaGetLastError());
}

}  // namespace rbo
