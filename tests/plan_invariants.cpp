// Host-side invariants of every launch plan the library can choose, checked
// over a grid of shapes without a GPU: shared memory within the opt-in limit
// of one CTA (227 KB), tensor-memory allocations a power of two in [32, 512]
// columns that hold the accumulators, every split-K range non-empty, padded
// batches covering the batch, TMA inner coordinates on 16-byte boundaries,
// and the scratch of every plan (and of every configuration the autotuner may
// install) within what grom_create allocates.  Built and run by
// tests/test_plan_invariants.py against libgrom.so.
#include <cstdio>
#include <vector>

#include "grom_internal.h"

using namespace grom;

static long g_fail = 0, g_checks = 0;
#define CHECK(cond, ...)                         \
  do {                                           \
    ++g_checks;                                  \
    if (!(cond)) {                               \
      if (g_fail < 20) {                         \
        std::printf("FAIL %s: ", #cond);         \
        std::printf(__VA_ARGS__);                \
        std::printf("\n");                       \
      }                                          \
      ++g_fail;                                  \
    }                                            \
  } while (0)

static const size_t SMEM_MAX = 232448;  // 227 KB opt-in dynamic shared memory per CTA

static bool tmem_ok(int cols) { return cols >= 32 && cols <= 512 && (cols & (cols - 1)) == 0; }

static void check_k1(int sm) {
  const int storages[] = {GROM_F64, GROM_F32X2, GROM_F32, GROM_BF16};
  for (int st : storages)
    for (int packed = 0; packed <= 1; ++packed)
      for (int64_t n : {1L, 2L, 3L, 17L, 64L, 100L, 511L, 512L, 1024L, 2048L, 4096L}) {
        if (n > grom_max_n(GROM_FORM_FULL, st)) continue;
        for (int64_t m : {0L, 1L, 64L, 129L}) {
          const K1Plan p = k1_plan(n, st, sm, packed, m);
          CHECK(p.smem <= SMEM_MAX, "K1 st %d packed %d n %ld m %ld smem %zu", st, packed, (long)n, (long)m, p.smem);
          CHECK(p.grid >= 1 && p.grid <= sm, "K1 grid %d", p.grid);
          CHECK(p.nb_max >= 1 && p.nb_max <= 8 && (p.nb_max & (p.nb_max - 1)) == 0, "K1 nb_max %d", p.nb_max);
          CHECK(p.rpc >= 1 && p.cpi * p.rpc >= p.m, "K1 rows per chunk n %ld", (long)n);
          // every row of a chunk lands in some consumer thread's registers
          const int planes = st == GROM_F32X2 ? 2 : 1;
          const int64_t rpr = k1_row_step(p, st);
          CHECK(k1_rmax(p.qm, planes) >= 1 && (p.rpc + rpr - 1) / rpr <= k1_rmax(p.qm, planes),
                "K1 rows per thread st %d packed %d n %ld", st, packed, (long)n);
          CHECK(p.row_bytes <= K1_MAX_ROW_BYTES && p.row_bytes % 16 == 0, "K1 row bytes %ld", (long)p.row_bytes);
          CHECK((int64_t)p.grid * (p.maxseg - 1) * p.cpi >= p.T - p.grid * p.cpi, "K1 segments n %ld", (long)n);
        }
      }
}

static void check_k2(int64_t n, int batch, int sm, int splits, size_t need) {
  const K2Plan p = k2_plan(n, batch, sm, splits);
  CHECK(p.smem <= SMEM_MAX, "K2 n %ld b %d smem %zu", (long)n, batch, p.smem);
  CHECK(tmem_ok(p.tmem_cols) && p.tmem_cols >= (p.btile <= 128 ? 4 * p.btile : 2 * p.btile), "K2 tmem %d btile %d",
        p.tmem_cols, p.btile);
  CHECK(p.splits >= 1 && p.splits <= n, "K2 splits %d n %ld", p.splits, (long)n);
  CHECK(p.btile % 16 == 0 && p.btile <= 256 && p.bp >= batch && p.bp - batch < p.btile, "K2 btile %d bp %ld b %d",
        p.btile, (long)p.bp, batch);
  CHECK(p.stages_a >= 2 && p.stages_b >= 2, "K2 stages");
  CHECK(p.np % 64 == 0 && p.np >= n, "K2 np");
  CHECK(k2_scratch_bytes(p) <= need, "K2 scratch n %ld b %d splits %d: %zu > %zu", (long)n, batch, splits,
        k2_scratch_bytes(p), need);
}

static void check_k2p(int64_t n, int64_t lp, int batch, int sm, int m, int ctas, size_t need) {
  const K2PPlan p = k2p_plan(n, lp, batch, sm, m, ctas);
  CHECK(p.ctas == 1 || p.ctas == 2, "K2P ctas %d", p.ctas);
  CHECK(ctas == 0 || p.ctas == ctas || (ctas == 2 && !k2p_pair_ok(lp) && p.ctas == 1), "K2P forced ctas %d -> %d",
        ctas, p.ctas);
  CHECK(p.ctas == 1 || (p.pblks >= 2 && k2p_pair_ok(lp)), "K2P pairs with %d blocks", p.pblks);
  // pairs: both CTAs of a pair tile take blocks 2q, 2q + 1 < pbs, so every
  // CTA tile has its own windows and direct partials in the scratch
  CHECK(p.ctas == 1 ? p.pbs == p.pblks : (p.pbs % 2 == 0 && p.pbs >= p.pblks && p.pbs <= p.pblks + 1),
        "K2P block stride %d (blocks %d, ctas %d)", p.pbs, p.pblks, p.ctas);
  CHECK(p.ctas == 1 || (p.grid % 2 == 0 && p.grid >= 2 && p.grid <= p.tiles && p.tiles % 2 == 0), "K2P pair grid %d",
        p.grid);
  if (p.ctas == 2 && n <= 1100 && batch % 61 == 1) {
    // the two CTAs of every pair tile cover each CTA tile exactly once, with
    // the tile numbering the finish kernel reads and in-range blocks and rows
    std::vector<char> seen((size_t)p.tiles, 0);
    bool ok = true;
    for (int t2 = 0; t2 < p.tiles / 2 && ok; ++t2)
      for (int rank = 0; rank < 2; ++rank) {
        int ct, pb, tile;
        int64_t i0, i1;
        k2p_pair_coords(t2, rank, p.col_tiles, p.pbs, p.m, n, ct, pb, i0, i1, tile);
        const int r = (int)(i0 / p.m);
        ok = ok && tile >= 0 && tile < p.tiles && !seen[(size_t)tile] && pb < p.pbs && ct < p.col_tiles &&
             i0 < n && i1 > i0 && i1 - i0 <= p.m && tile == (r * p.pbs + pb) * p.col_tiles + ct;
        if (ok) seen[(size_t)tile] = 1;
      }
    for (char c : seen) ok = ok && c;
    CHECK(ok, "K2P pair tiles n %ld b %d m %d", (long)n, batch, p.m);
  }
  CHECK(p.smem <= SMEM_MAX, "K2P n %ld b %d m %d smem %zu", (long)n, batch, p.m, p.smem);
  CHECK(p.stages >= 2, "K2P stages %d", p.stages);
  CHECK(tmem_ok(p.tmem_cols) && p.tmem_cols >= 4 * p.btile, "K2P tmem %d", p.tmem_cols);
  CHECK(p.m >= 8 && p.m <= 32 && (m == 0 || p.m == m), "K2P m %d forced %d", p.m, m);
  CHECK((int64_t)p.ranges * p.m >= n && (int64_t)(p.ranges - 1) * p.m < n, "K2P ranges");
  CHECK(p.tiles == p.ranges * p.pbs * p.col_tiles && p.grid >= 1 && p.grid <= sm, "K2P tiles");
  CHECK((int64_t)p.pblks * 128 >= p.lp && p.lp % 64 == 0, "K2P position blocks lp %ld", (long)p.lp);
  CHECK(p.wrows == p.m + 127 && p.wpitch == p.btile + 1, "K2P window");
  CHECK(p.btile % 16 == 0 && p.btile <= 128 && p.bp >= batch && p.bp - batch < p.btile, "K2P btile");
  CHECK(k2p_scratch_bytes(p) <= need, "K2P scratch n %ld b %d m %d: %zu > %zu", (long)n, batch, p.m,
        k2p_scratch_bytes(p), need);
}

static void check_k3t(int64_t n, int64_t r, int form, int batch, int sm, int s1, int s2, size_t need) {
  const K3TPlan p = k3t_plan(n, r, form, batch, sm, s1, s2);
  CHECK(p.smem <= SMEM_MAX && p.stages >= 2, "K3T smem %zu stages %d", p.smem, p.stages);
  CHECK(tmem_ok(p.tmem_cols) && p.tmem_cols >= 2 * p.btile, "K3T tmem %d", p.tmem_cols);
  CHECK(p.k1 % 64 == 0 && p.k2 % 64 == 0 && p.rp % 64 == 0, "K3T K extents (TMA x in 64-element blocks)");
  CHECK(p.s1 >= 1 && p.s1 <= p.s1_max && p.s1 <= p.k1 / 64, "K3T s1 %d (max %d, K blocks %ld)", p.s1, p.s1_max,
        (long)(p.k1 / 64));
  CHECK(p.s2 >= 1 && p.s2 <= p.s2_max && p.s2 <= p.k2 / 64, "K3T s2 %d (max %d, K blocks %ld)", p.s2, p.s2_max,
        (long)(p.k2 / 64));
  CHECK((s1 == 0 || p.s1 == s1) && (s2 == 0 || p.s2 == s2), "K3T forced splits (%d, %d) -> (%d, %d)", s1, s2, p.s1,
        p.s2);
  CHECK(p.btile % 16 == 0 && p.btile <= 128 && p.bp >= batch && p.bp - batch < p.btile, "K3T btile");
  // projection kernel: nseg accumulators of 2 btile columns in tensor memory
  CHECK(p.smem_p <= SMEM_MAX && p.stages_p >= 2, "K3T projection smem %zu stages %d", p.smem_p, p.stages_p);
  CHECK(tmem_ok(p.tmem_p) && p.tmem_p >= p.nseg * 2 * p.btile, "K3T projection tmem %d (nseg %d btile %d)", p.tmem_p,
        p.nseg, p.btile);
  CHECK(p.jtiles * 128 >= p.rp && p.ctiles <= K3T_MAX_CTILES, "K3T tiles %d x %d", p.jtiles, p.ctiles);
  // the counters sit at the start of the scratch, one region per (n, r)
  CHECK(k3t_counter_bytes(p) == k3t_counter_bytes(k3t_plan(n, r, form, 16, sm)), "K3T counter region moves");
  CHECK(k3t_scratch_bytes(p) <= need, "K3T scratch n %ld r %ld b %d (%d, %d): %zu > %zu", (long)n, (long)r, batch,
        p.s1, p.s2, k3t_scratch_bytes(p), need);
}

// Every configuration grom_tune_space offers, applied to the plans.
static std::vector<grom_tuning> space(int form, int layout, int64_t n, int64_t r, int max_batch, int batch, int sm) {
  const int cnt = grom_tune_space(form, GROM_BF16, layout, (int)n, (int)r, max_batch, batch, sm, nullptr, 0);
  std::vector<grom_tuning> v(cnt > 0 ? cnt : 0);
  if (cnt > 0) grom_tune_space(form, GROM_BF16, layout, (int)n, (int)r, max_batch, batch, sm, v.data(), cnt);
  return v;
}

int main() {
  for (int sm : {132, 148, 152}) {
    check_k1(sm);
    for (int64_t n : {1L, 2L, 3L, 17L, 64L, 96L, 129L, 200L, 300L, 512L, 1024L, 2048L}) {
      const int64_t lp = k1_plan(n, GROM_BF16, sm, 1).lp;
      for (int max_batch : {1, 8, 16, 40, 130, 256, 1024, 1300}) {
        const size_t need2 = k2_scratch_need(n, max_batch, sm), need2p = k2p_scratch_need(n, lp, max_batch, sm);
        for (int b = 1; b <= max_batch; b += (b < 300 ? 1 : 37)) {
          check_k2(n, b, sm, 0, need2);
          for (int ctas = 0; ctas <= 2; ++ctas) check_k2p(n, lp, b, sm, 0, ctas, need2p);
          if (b % 16 == 1 || b == max_batch) {  // one batch per bucket: the tune space
            for (const grom_tuning& t : space(GROM_FORM_FULL, GROM_LAYOUT_DENSE, n, 0, max_batch, b, sm))
              if (t.kernel == GROM_KERNEL_TENSOR) check_k2(n, b, sm, t.split_a, need2);
            for (const grom_tuning& t : space(GROM_FORM_FULL, GROM_LAYOUT_SKEW_PACKED, n, 0, max_batch, b, sm))
              if (t.kernel == GROM_KERNEL_TENSOR) check_k2p(n, lp, b, sm, t.tile_m, t.split_b, need2p);
          }
        }
        for (int form : {GROM_FORM_CP, GROM_FORM_CP_SKEW})
          for (int64_t r : {1L, 5L, 64L, 129L, 512L, 1024L}) {
            const size_t need3 = k3t_scratch_need(n, r, form, max_batch, sm);
            for (int b = 1; b <= max_batch; b += (b < 300 ? 3 : 61)) {
              check_k3t(n, r, form, b, sm, 0, 0, need3);
              if (b % 16 == 1)
                for (const grom_tuning& t : space(form, GROM_LAYOUT_DENSE, n, r, max_batch, b, sm))
                  if (t.kernel == GROM_KERNEL_TENSOR) check_k3t(n, r, form, b, sm, t.split_a, t.split_b, need3);
            }
          }
      }
    }
  }
  std::printf("%ld checks, %ld failed\n", g_checks, g_fail);
  return g_fail == 0 ? 0 : 1;
}
