// Mixed-precision Lanczos phase A of the batch (z = sigma_j H U_j -
// ratio_j U_{j-1}, alpha_j = sigma_j Re <U_j, z>) over tiles of 256 radial
// columns x kTileRows partial waves, with the rows of every operand staged
// into shared memory by bulk asynchronous copies (cp.async.bulk, completion
// on an mbarrier).
//
// Included by tdse_batch.cu inside its anonymous namespace (it uses the
// engine's device descriptors, field table and reduction slots).
//
// Why tiles: the register walker gives each warp a 32-column strip and walks
// it down the partial waves, so every row of every array is read in 256-byte
// pieces (128 for the FP32 diagonal) scattered over the whole batch, with the
// stencil's two halo columns on each side in sectors shared with other
// strips.  Here the 8 warps of a CTA walk one 256-column block together: a
// row of the operand (with its halo), of the diagonal and of the epilogue
// operand arrives as one contiguous 2 KB (1 KB) piece per array, issued by one
// thread as a bulk copy that lands in a ring of D row slots while the block
// computes the rows before it.
//
// Alignment: a bulk copy moves 16-byte-aligned runs of whole 16-byte units.
// Rows start wherever (r N) lands (N may be odd), so each piece is widened to
// the enclosing 16-byte run and a thread indexes its value from the remainder
// in shared memory.  The widened run stays inside the instance's region: every
// array of a region starts on a 256-byte boundary, and a run never starts
// before its row's first element nor ends more than 15 bytes after its last.
//
// Reductions: a tile's partial is the fixed-order block sum of the threads'
// pair sums (thread = column, its rows in order); the last tile of an
// instance to finish adds the instance's tile partials in tile order.  Tiles
// depend only on the instance, so results do not depend on the batch or the
// schedule (bitwise).
//
// Waits: the consumers wait on the slot's mbarrier, the producer's copies
// being the only thing that completes it; every wait gives up after
// kTileSpins polls, sets kStatusTimeout in the status word (reported by the
// next synchronising call) and carries on with what the slot holds, so the
// block's barriers stay uniform and the kernel ends.

constexpr int kTileCols = 256;               // radial columns of a tile = threads of a block
constexpr int kTileRows = TDSE_TILE_ROWS;    // partial waves of a tile
constexpr int kTileThreads = kTileCols;       // consumer threads: one per column
constexpr long long kTileSpins = 1LL << 26;  // polls of an mbarrier before giving up
// Slot layout (bytes) per MODE (see below): the operand row with its two halo
// columns on each side (two parts, hi and lo, in MODE 0), the diagonal row and
// the epilogue row (two parts in MODE 1), each with room for 16 bytes of
// alignment slack.
constexpr int kOpBytes = ((kTileCols + 4) * 8 + 16 + 127) / 128 * 128;
constexpr int kDgBytes = (kTileCols * 4 + 16 + 127) / 128 * 128;
constexpr int kEpBytes = (kTileCols * 8 + 16 + 127) / 128 * 128;
template <int MODE>
struct SlotLayout {
  static constexpr int op0 = 0;
  static constexpr int op1 = kOpBytes;                              // MODE 0 only
  static constexpr int dg = (MODE == 0 ? 2 : 1) * kOpBytes;
  static constexpr int ep0 = dg + kDgBytes;                         // MODE 1, 2
  static constexpr int ep1 = ep0 + kEpBytes;                        // MODE 1 only
  static constexpr int bytes = MODE == 0 ? dg + kDgBytes : (MODE == 1 ? ep1 + kEpBytes : ep0 + kEpBytes);
};
constexpr int kTileBarBytes = 512;           // the ring's full and empty mbarriers, ahead of the slots
constexpr int kTileMaxDepth = 24;
constexpr int kTileConsumerWarps = kTileThreads / 32;
constexpr int kTileBlock = kTileThreads + 32;   // 8 consumer warps and one producer warp

template <int MODE, int D>
constexpr int tile_smem_bytes() { return kTileBarBytes + D * SlotLayout<MODE>::bytes; }

__device__ __forceinline__ unsigned tsmem(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tsmem(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tsmem(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(tsmem(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bytes (a multiple of 16) from global src (16-byte aligned) to shared dst
// (16-byte aligned), completing on bar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tsmem(dst)),
               "l"(src), "r"(bytes), "r"(tsmem(bar))
               : "memory");
}

// Wait for phase `parity` of bar, at most kTileSpins polls; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  for (long long s = 0; s < kTileSpins; ++s)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// The widened 16-byte run holding elements [e0, e1) of an array of esz-byte
// elements; the copy's source, byte count and the offset of element e0 in it.
struct Run {
  const char *src;
  unsigned bytes, off;
};
__device__ __forceinline__ Run run_of(const void *base, long long e0, long long e1, int esz) {
  const uintptr_t a = (uintptr_t)base + (uintptr_t)(e0 * esz);
  const uintptr_t b = (uintptr_t)base + (uintptr_t)(e1 * esz);
  const uintptr_t a0 = a & ~(uintptr_t)15, b1 = (b + 15) & ~(uintptr_t)15;
  return Run{reinterpret_cast<const char *>(a0), (unsigned)(b1 - a0), (unsigned)(a - a0)};
}

// Where tile gt of a chunk list lies: instance, first column, rows [l0, l1).
struct TileAt {
  int inst, lt, c0, l0, l1;
};
__device__ __forceinline__ TileAt tile_at(const BatchDev &B, const ChunkList &cl, int gt, int &p) {
  while (cl.cpre[p + 1] <= gt) ++p;
  TileAt t;
  t.inst = cl.act[p];
  t.lt = gt - cl.cpre[p];
  const BatchInst &I = B.inst[t.inst];
  const int nr = (I.L + kTileRows) / kTileRows;    // ceil((L + 1) / kTileRows)
  const int c = t.lt / nr, r = t.lt - c * nr;
  t.c0 = c * kTileCols;
  t.l0 = r * kTileRows;
  t.l1 = min(t.l0 + kTileRows, I.L + 1);
  return t;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tsmem(bar)) : "memory");
}
__device__ __forceinline__ void consumers_sync() {   // the 8 consumer warps only (named barrier 1)
  asm volatile("bar.sync 1, %0;" ::"n"(kTileThreads) : "memory");
}

// One tile's arrays, read once per tile from the instance's descriptor.
// MODE 0: the operand is the split of psi (hi + lo, j = 0); MODE 1: the
// operand is U_1 and the epilogue U_0 = the split of psi; MODE 2: the operand
// is U_j and the epilogue U_{j-1}.
template <int MODE>
struct TileArrays {
  const float2 *x0, *x1;    // operand (parts)
  const float *dg;          // FP32 diagonal
  const float2 *e0, *e1;    // epilogue (parts)
  long long N;
  int L;
};

template <int MODE>
__device__ __forceinline__ TileArrays<MODE> tile_arrays(const BatchInst &I, int j) {
  TileArrays<MODE> a;
  const long long G = (long long)I.N * (I.L + 1);
  a.N = I.N;
  a.L = I.L;
  a.x0 = MODE == 0 ? I.hi : I.mwork + (long long)j * G;
  a.x1 = I.lo;
  a.dg = I.diagf;
  a.e0 = MODE == 1 ? I.hi : I.mwork + (long long)(j - 1) * G;
  a.e1 = I.lo;
  return a;
}

// Issue the copies of one row item (row `row` of a tile whose first column is
// c0 and whose rows are [l0, l1)) into `slot`: the operand row with its halo
// for every row in [0, L], the diagonal and epilogue rows for rows in
// [l0, l1) only; rows outside [0, L] complete the barrier with no bytes.
template <int MODE>
__device__ __forceinline__ void tile_issue(const TileArrays<MODE> &A, int c0, int l0, int l1, int row,
                                           unsigned char *slot, unsigned long long *bar, unsigned *offs) {
  using SL = SlotLayout<MODE>;
  unsigned bytes = 0;
  Run op0{}, op1{}, dg{}, ep0{}, ep1{};
  const bool have = row >= 0 && row <= A.L;
  const bool body = row >= l0 && row < l1;
  if (have) {
    const long long rb = (long long)row * A.N;
    const long long cs = max(c0 - 2, 0), ce = min((long long)c0 + kTileCols + 2, A.N);
    op0 = run_of(A.x0, rb + cs, rb + ce, 8);
    bytes += op0.bytes;
    if (MODE == 0) {
      op1 = run_of(A.x1, rb + cs, rb + ce, 8);
      bytes += op1.bytes;
    }
    if (body) {
      const long long de = min((long long)c0 + kTileCols, A.N);
      dg = run_of(A.dg, rb + c0, rb + de, 4);
      bytes += dg.bytes;
      if (MODE >= 1) {
        ep0 = run_of(A.e0, rb + c0, rb + de, 8);
        bytes += ep0.bytes;
      }
      if (MODE == 1) {
        ep1 = run_of(A.e1, rb + c0, rb + de, 8);
        bytes += ep1.bytes;
      }
    }
  }
  // where the first element of each part sits in its run (published with the
  // arrival below: the consumers read them after their wait on the barrier)
  offs[0] = op0.off;
  offs[1] = op1.off;
  offs[2] = dg.off;
  offs[3] = ep0.off | (ep1.off << 8);
  // the async proxy writes the slot next: order it after the consumers' reads of it
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect(bar, bytes);
  if (have) {
    bulk_g2s(slot + SL::op0, op0.src, op0.bytes, bar);
    if (MODE == 0) bulk_g2s(slot + SL::op1, op1.src, op1.bytes, bar);
    if (body) {
      bulk_g2s(slot + SL::dg, dg.src, dg.bytes, bar);
      if (MODE >= 1) bulk_g2s(slot + SL::ep0, ep0.src, ep0.bytes, bar);
      if (MODE == 1) bulk_g2s(slot + SL::ep1, ep1.src, ep1.bytes, bar);
    }
  }
}

// Staged row as an array indexed by global column: element c of the row that
// was copied from element rb + c_first of base sits at part + off + esz (c - c_first).
template <typename T>
__device__ __forceinline__ const T *staged_row(const unsigned char *part, const T *base, long long rb,
                                               long long c_first) {
  const unsigned off = (unsigned)(((uintptr_t)(base + rb + c_first)) & 15);
  return reinterpret_cast<const T *>(part + off) - c_first;
}

// Lanczos phase A (mixed) over this block's tiles.  Warps 0..7 compute (thread
// = column); warp 8 lane 0 issues the row copies D items ahead.  Items run
// through a ring of D slots: full[s] completes when an item's bytes have
// landed, empty[s] when all 8 consumer warps are done with it.  A tile with
// rows [l0, l1) is the item sequence l0 - 1, l0, ..., l1 (one row of l-halo
// on each side); a consumer holds rows l - 1, l, l + 1 while it computes row l.
template <int ST, int MODE, int D>
__global__ void __launch_bounds__(kTileBlock, 3)
    bt_lanczos_a_mixed_tile(BatchDev B, ChunkList cl, int j) {
  static_assert(D >= 3 && D <= kTileMaxDepth, "ring depth");
  using SL = SlotLayout<MODE>;
  extern __shared__ __align__(128) unsigned char tile_smem[];
  __shared__ double s_red[kTileConsumerWarps];
  __shared__ unsigned s_last;
  __shared__ unsigned s_offs[kTileMaxDepth][4];   // per slot: offsets of its parts' first elements
  unsigned long long *full = reinterpret_cast<unsigned long long *>(tile_smem);
  unsigned long long *empty = full + kTileMaxDepth;
  unsigned char *slots = tile_smem + kTileBarBytes;
  const int tid = threadIdx.x;
  // this block's tiles: a balanced contiguous range of the list
  const unsigned T = (unsigned)cl.total, nb = gridDim.x, b = blockIdx.x;
  const unsigned q = T / nb, rem = T - q * nb;
  const int g0 = (int)(b * q + min(b, rem)), g1 = g0 + (int)(q + (b < rem ? 1u : 0u));
  if (g0 >= g1) return;   // uniform over the block
  if (tid == 0) {
    for (int s = 0; s < D; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kTileConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();   // the last barrier the producer warp takes part in
  bool timed_out = false;

  if (tid >= kTileThreads) {
    // ---- producer warp -----------------------------------------------------
    if (tid == kTileThreads) {
      long long item = 0;
      int p = find_owner(cl, g0);
      for (int gt = g0; gt < g1; ++gt) {
        const TileAt t = tile_at(B, cl, gt, p);
        const TileArrays<MODE> A = tile_arrays<MODE>(B.inst[t.inst], j);
        for (int row = t.l0 - 1; row <= t.l1; ++row, ++item) {
          const int s = (int)(item % D);
          if (item >= D && !mbar_wait(&empty[s], (unsigned)((item / D - 1) & 1))) timed_out = true;
          tile_issue<MODE>(A, t.c0, t.l0, t.l1, row, slots + (size_t)s * SL::bytes, &full[s], s_offs[s]);
        }
      }
    }
    if (timed_out) atomicOr(B.status, kStatusTimeout);
    return;
  }

  // ---- consumer warps --------------------------------------------------------
  const int lane = tid & 31, warp = tid >> 5;
  // ring positions, advanced incrementally (no division by D): the next slot
  // to wait for and its phase parity, and the next slot to free
  int ws = 0, fs = 0;
  unsigned wph = 0;
  auto wait_item = [&]() -> int {
    const int s = ws;
    if (!mbar_wait(&full[s], wph)) timed_out = true;
    if (++ws == D) {
      ws = 0;
      wph ^= 1u;
    }
    return s;
  };
  auto release = [&]() {   // this warp is done with the oldest item it holds
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[fs]);
    if (++fs == D) fs = 0;
  };
  // a staged part as an array over the global column: element c sits at
  // part + off + esz (c - first column of the copy)
  auto part = [&](int s, int p, unsigned off, long long cfirst) -> const unsigned char * {
    return slots + (size_t)s * SL::bytes + p + off - 8 * cfirst;
  };
  int cp = find_owner(cl, g0);
  for (int gt = g0; gt < g1; ++gt) {
    const TileAt t = tile_at(B, cl, gt, cp);
    const BatchInst &I = B.inst[t.inst];
    LanczosScalars *ls = B.ls + t.inst;
    const int N = I.N, L = I.L;
    const int jj = t.c0 + tid;
    const bool active = jj < N;
    const double sigd = ls->sigma[j];
    const float sig = (float)sigd;
    const float cprev = (j > 0) ? (float)ls->ratio[j] : 0.f;
    const float c1 = (float)I.c1, c2 = (float)I.c2;
    const float E = (float)field_of(B, t.inst);
    const float Er = active ? E * I.rjf[jj] : 0.f;
    float2 *z = I.mwork;
    const long long cs = max(t.c0 - 2, 0);
    const bool ok_m1 = jj >= 1, ok_p1 = jj + 1 < N, ok_m2 = jj >= 2, ok_p2 = jj + 2 < N;
    const float2 zero = make_float2(0.f, 0.f);
    // operand row of slot s as arrays over the global column (hi / lo parts in MODE 0)
    auto opr = [&](int s, int which) -> const float2 * {
      return reinterpret_cast<const float2 *>(part(s, which ? SL::op1 : SL::op0, s_offs[s][which], cs));
    };
    auto center = [&](int s) -> float2 {
      if (MODE == 0) {
        const float2 h = opr(s, 0)[jj], lw = opr(s, 1)[jj];
        return make_float2(lw.x + h.x, lw.y + h.y);
      }
      return opr(s, 0)[jj];
    };
    PairSum acc;
    const int sprev = wait_item();
    float2 vp = (t.l0 > 0 && active) ? center(sprev) : zero;
    int scur = wait_item();
    const float2 *h = opr(scur, 0);
    const float2 *w = MODE == 0 ? opr(scur, 1) : nullptr;
    float2 vc = active ? center(scur) : zero;
    float a_cur = I.kappaf[t.l0] * Er;
    float2 *zrow = z + (long long)t.l0 * N + jj;
    for (int l = t.l0; l < t.l1; ++l) {
      const int snext = wait_item();
      const float2 *hn = opr(snext, 0);
      const float2 *wn = MODE == 0 ? opr(snext, 1) : nullptr;
      float2 vn = zero;
      if (l < L && active) {
        vn = hn[jj];
        if (MODE == 0) {
          const float2 lw = wn[jj];
          vn = make_float2(lw.x + vn.x, lw.y + vn.y);
        }
      }
      const float a_next = I.kappaf[l + 1] * Er;
      if (active) {
        // a - c part by part (the difference form of the Laplacian), zero beyond the box
        const float2 hc = h[jj];
        const float2 lc = MODE == 0 ? w[jj] : zero;
        auto dif = [&](int cc, bool ok) -> float2 {
          if (MODE == 0) {
            const float2 ha = ok ? h[cc] : zero, la = ok ? w[cc] : zero;
            float2 d = make_float2(la.x - lc.x, la.y - lc.y);
            d.x += ha.x - hc.x;
            d.y += ha.y - hc.y;
            return d;
          }
          const float2 a = ok ? h[cc] : zero;
          return make_float2(1.f * (a.x - hc.x), 1.f * (a.y - hc.y));
        };
        const float2 d1m = dif(jj - 1, ok_m1), d1p = dif(jj + 1, ok_p1);
        const unsigned eo = s_offs[scur][3];
        const float dg = reinterpret_cast<const float *>(part(scur, SL::dg, s_offs[scur][2], 0) +
                                                         4 * (long long)tid)[0];
        float tx = c1 * (d1m.x + d1p.x);
        float ty = c1 * (d1m.y + d1p.y);
        if (ST == 5) {
          const float2 d2m = dif(jj - 2, ok_m2), d2p = dif(jj + 2, ok_p2);
          tx = fmaf(c2, d2m.x + d2p.x, tx);
          ty = fmaf(c2, d2m.y + d2p.y, ty);
        }
        tx = fmaf(dg, vc.x, tx);
        ty = fmaf(dg, vc.y, ty);
        tx = fmaf(a_cur, vp.x, tx);
        ty = fmaf(a_cur, vp.y, ty);
        tx = fmaf(a_next, vn.x, tx);
        ty = fmaf(a_next, vn.y, ty);
        float2 o = make_float2(sig * tx, sig * ty);
        if (MODE > 0) {
          float2 up = reinterpret_cast<const float2 *>(part(scur, SL::ep0, eo & 255u, 0))[tid];
          if (MODE == 1) {
            const float2 lw = reinterpret_cast<const float2 *>(part(scur, SL::ep1, eo >> 8, 0))[tid];
            up = make_float2(up.x + lw.x, up.y + lw.y);
          }
          o.x = fmaf(-cprev, up.x, o.x);
          o.y = fmaf(-cprev, up.y, o.y);
        }
        *zrow = o;
        acc.add(fmaf(vc.x, o.x, vc.y * o.y));
      }
      vp = vc;
      vc = vn;
      a_cur = a_next;
      release();          // the item of row l - 1
      scur = snext;
      h = hn;
      w = wn;
      zrow += N;
    }
    release();            // rows l1 - 1 and l1
    release();
    // the tile's partial (fixed order: lanes by the xor tree, warps in order),
    // then the instance's sum if this was its last tile
    double v = warp_sum(acc.value());
    if (lane == 0) s_red[warp] = v;
    consumers_sync();
    if (tid == 0) {
      double sm = 0.0;
      for (int w2 = 0; w2 < kTileConsumerWarps; ++w2) sm += s_red[w2];
      I.partial[t.lt] = sm;
      __threadfence();
      s_last = (atomicAdd(&B.ticket[t.inst], 1u) == (unsigned)(I.nchunk - 1)) ? 1u : 0u;
    }
    consumers_sync();
    if (s_last) {
      __threadfence();
      double sm = 0.0;
      for (int c = tid; c < I.nchunk; c += kTileThreads) sm += __ldcg(&I.partial[c]);
      sm = warp_sum(sm);
      if (lane == 0) s_red[warp] = sm;
      consumers_sync();
      if (tid == 0) {
        double tot = 0.0;
        for (int w2 = 0; w2 < kTileConsumerWarps; ++w2) tot += s_red[w2];
        ls->alpha[j] = tot * sigd;
        ls->acoef[j] = -(tot * sigd) * sigd;
        B.ticket[t.inst] = 0u;
      }
    }
    consumers_sync();
  }
  if (timed_out) atomicOr(B.status, kStatusTimeout);
}
