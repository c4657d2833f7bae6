// Host planner: expands the tile DAG of the tiled Cholesky and of the
// two-phase selected inversion into fine-block tasks, then orders them by a
// critical-path-first list schedule.
//
// Tile-level method (sTiles selected inversion, arXiv 2504.19171):
//   factor  (Sec. III)       for k: L_kk = POTRF(A_kk); L_ik = A_ik L_kk^{-T};
//                            A_ij -= L_ik L_jk^T for i >= j in struct(k)
//   phase 1 (Algorithm 2)    Linv_ii = L_ii^{-1} ("TRSM against I");
//                            Sigma_ii^0 = Linv_ii^T Linv_ii (LAUUM);
//                            U_ki = L_ki Linv_ii (TRMM), k in struct(i)
//   phase 2 (Algorithm 3,    for i descending: Sigma_ji = -sum_k S_jk U_ki,
//            Sec. III-A)     j in struct(i) (S_jk = Sigma_jk or Sigma_kj^T);
//                            Sigma_ii = Sigma_ii^0 - sum_k Sigma_ki^T U_ki
// Each tile operation is split over FB x FB output blocks so that one b x b
// tile operation occupies many SMs at once; the per-block work is a K-loop
// over contiguous panels of other tiles (a "segment").
//
// The factorization runs at fine-block granularity in right-looking order
// (every b x b POTRF/TRSM/SYRK/GEMM decomposes exactly into FB-block POTRF,
// TRSM and GEMM updates), which keeps the critical path at about three small
// block operations per FB columns. Updates into one block are applied by a
// chain of tasks in increasing source column, so a block's terms are always
// summed in the same order whatever the schedule (bit-reproducible results).
// Batches (build_batch_plan) merge several matrices' tables under one list
// schedule; request-server templates (build_serve_template) add one OP_PREP
// task per tile column that builds A on the device.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <functional>
#include <queue>

#include "../../include/stiles.h"

namespace stiles {
namespace {

// Cost model for the list schedule: one SM of a GB300 at about 1.9 GHz with
// 2 FP64 FMA per clock does ~7.6 flop/ns, shared by the kCtasPerSm workers
// that run on it; plus a per-task overhead.
constexpr double kFlopPerNs = 7.6 / kCtasPerSm;
constexpr double kTaskOverheadNs = 2500.0;
constexpr double kSweepStepNs = 120.0;  // one step of an in-shared-memory triangular sweep

struct Builder {
  Shape s;
  Layout L;
  PlanKind kind;
  Plan* out;
  // per emitted task (emission order is topological)
  std::vector<Task> tasks;
  std::vector<double> cost;
  // segments, waits and signalled counters of task t: [off[t], off[t+1]) of each flat array
  std::vector<Seg> fsegs;
  std::vector<Wait> fwaits;
  std::vector<int32_t> fsigs;
  std::vector<int64_t> seg_off{0}, wait_off{0}, sig_off{0};
  // counters (their writers, in emission order, are the tasks that list them in fsigs)
  std::vector<char> chain;  // 1: writers strictly ordered
  double flops = 0;
  double flops_lowered = 0;  // algorithmic flops of the reduced-precision block products
  bool sym_block = false;    // the next emitted task updates a symmetric diagonal block (m^2 k per term)
  long long tile_gemms = 0;
  int ndiag = 0;

  bool serve = false;                // emit OP_PREP tasks (request server template)
  std::vector<int32_t> prep_ctr;     // serve: per tile column, signalled by its PREP task

  Builder(const Shape& sh, PlanKind k, Plan* o) : s(sh), L(sh), kind(k), out(o) {}

  int32_t newctr(bool is_chain) {
    chain.push_back(is_chain ? 1 : 0);
    return (int32_t)chain.size() - 1;
  }

  int emit(Task t, std::vector<Seg> segs, std::vector<Wait> waits, std::vector<int32_t> sigs, double epi_ns) {
    double f = 0;
    for (const Seg& g : segs) f += 2.0 * t.m * t.n * g.k;
    // the same products under the counting convention (a symmetric diagonal
    // block's update counts m^2 k, like SYRK), for the reduced-precision share
    if (t.prec != PREC_FP64) flops_lowered += sym_block ? 0.5 * f : f;
    sym_block = false;
    if (t.pmode == PM_TRI3) f *= 0.75;
    if (t.prec == PREC_EMU64) f /= 10.0;   // order of the emulated-FP64 speed-up per block
    if (t.prec == PREC_FP32X) f /= 25.0;
    int id = (int)tasks.size();
    tasks.push_back(t);
    // parts run side by side on different CTAs
    cost.push_back(kTaskOverheadNs + f / kFlopPerNs / t.parts +
                   epi_ns / (t.pmode == PM_ROWS2 ? 2 : t.pmode == PM_ROWS4 ? 4 : 1));
    fsegs.insert(fsegs.end(), segs.begin(), segs.end());
    seg_off.push_back((int64_t)fsegs.size());
    fwaits.insert(fwaits.end(), waits.begin(), waits.end());
    wait_off.push_back((int64_t)fwaits.size());
    fsigs.insert(fsigs.end(), sigs.begin(), sigs.end());
    sig_off.push_back((int64_t)fsigs.size());
    return id;
  }

  static Task blank(uint8_t op, int m, int n) {
    Task t{};
    t.out = t.cin = t.aux = -1;
    t.op = op;
    t.m = (int16_t)m;
    t.n = (int16_t)n;
    t.diag = -1;
    t.parts = 1;
    t.pmode = PM_FULL;
    t.prec = PREC_FP64;
    return t;
  }

  // Divide a block task among CTAs; a mode that would leave a part empty
  // (blocks of at most 32 rows or columns) falls back to one part.
  static void split(Task& t, uint8_t mode) {
    if (mode == PM_ROWS2 && t.m > 32) { t.pmode = PM_ROWS2; t.parts = 2; }
    else if (mode == PM_ROWS4 && t.m > 48) { t.pmode = PM_ROWS4; t.parts = 4; }
    else if (mode == PM_ROWS4 && t.m > 32) { t.pmode = PM_ROWS2; t.parts = 2; }
    else if (mode == PM_QUAD4 && t.m > 32 && t.n > 32) { t.pmode = PM_QUAD4; t.parts = 4; }
    else if (mode == PM_TRI3 && t.m > 32 && t.m == t.n) { t.pmode = PM_TRI3; t.parts = 3; }
    else if (mode == PM_ROWS8 && t.m > 8 && t.m <= 32) { t.pmode = PM_ROWS8; t.parts = (uint8_t)((t.m + 7) / 8); }
    else if (mode == PM_TRI16 && t.m > 16 && t.m <= 32 && t.m == t.n) { t.pmode = PM_TRI16; t.parts = 3; }
    else if (mode == PM_QUAD16 && t.m <= 32 && t.n > 16 && t.n <= 32) {
      t.pmode = PM_QUAD16;
      t.parts = t.m > 16 ? 4 : 2;  // parts 2 and 3 are the lower row of quadrants
    }
  }

  // Parts of an off-diagonal phase-2 block task (tuning bits 2-3).
  void split_p2(Task& t) const {
    const int mode = tune_p2_split(s.tune);
    if (mode == 0) split(t, PM_QUAD4);
    else if (mode == 1) split(t, PM_ROWS2);
  }

  // Mark a bulk product task with the plan's reduced precision. The tensor-
  // core digit products work on sub-tiles of at most 32 x 32 (four digit
  // planes of 32 rows fill the 128 rows of one MMA): blocks that are not
  // already split that way run as a grid of such tiles.
  void lower_precision(Task& t) const {
    if (s.prec == PREC_FP64) return;
    t.prec = (uint8_t)s.prec;
    if (t.pmode != PM_QUAD4 && t.pmode != PM_TRI3) {
      const int pr = t.m > 32 ? 2 : 1, pc = t.n > 32 ? 2 : 1;
      t.pmode = PM_TILE32;
      t.parts = (uint8_t)(pr * pc);
    }
  }

  static Seg seg(int64_t a, int lda, int64_t b, int ldb, int k, bool ta, bool tb) {
    Seg g;
    g.a = a; g.b = b; g.lda = lda; g.ldb = ldb; g.k = k;
    g.trans = (ta ? 1 : 0) | (tb ? 2 : 0);
    return g;
  }

  // ------------------------------------------------------------ factor ----
  // Fine rows are (tile, block row) pairs; a fine column is (tile k, block c).
  // Counter ids of L blocks: lctr[k][i-slot][r][c] flattened.
  std::vector<int32_t> lctr;       // per L block (lower pattern)
  std::vector<int64_t> lctr_base;  // per (i,k) tile: first index into lctr, or -1
  std::vector<int32_t> lfinal;     // per L block: number of writers (updates + final)
  std::vector<int32_t> colfinal;   // fused: per tile column, counter of "L column final"
  std::vector<int32_t> coljoin;    // fused: per tile column, the join task's counter (one writer)
  std::vector<int32_t> colblocks;  // fused: number of L blocks per tile column

  int tile_slot(int i, int k) const {  // 0 = diag, 1..w = band, w+1 = arrow
    if (i == k) return 0;
    if (i == s.nt) return s.w + 1;
    return i - k;
  }
  int64_t& tbase(int i, int k) { return lctr_base[(size_t)k * (s.w + 2) + tile_slot(i, k)]; }
  int32_t lidx(int i, int k, int r, int c) { return (int32_t)(tbase(i, k) + (int64_t)r * L.nblk(k) + c); }

  void alloc_lblocks() {
    int cols = L.last() + 1;
    lctr_base.assign((size_t)cols * (s.w + 2), -1);
    std::vector<int> st;
    int64_t nb = 0;
    for (int k = 0; k < cols; ++k) {
      tbase(k, k) = nb;
      nb += (int64_t)L.nblk(k) * L.nblk(k);
      L.structure(k, st);
      for (int i : st) {
        tbase(i, k) = nb;
        nb += (int64_t)L.nblk(i) * L.nblk(k);
      }
    }
    lctr.assign(nb, -1);
    lfinal.assign(nb, 0);
  }

  void build_factor() {
    alloc_lblocks();
    std::vector<int> st, stk;
    int cols = L.last() + 1;
    // count writers: updates per block + 1 final; and create chain counters
    if (kind == PLAN_FUSED) {
      colfinal.resize(cols);
      colblocks.assign(cols, 0);
      for (int k = 0; k < cols; ++k) colfinal[k] = newctr(false);
    }
    for (int k = 0; k < cols; ++k) {
      L.structure(k, st);
      std::vector<int> rows_i;  // tiles in this column: k and struct(k)
      rows_i.push_back(k);
      for (int i : st) rows_i.push_back(i);
      for (int i : rows_i)
        for (int r = 0; r < L.nblk(i); ++r)
          for (int c = 0; c < L.nblk(k); ++c) {
            if (i == k && r < c) continue;
            lctr[lidx(i, k, r, c)] = newctr(true);
            if (kind == PLAN_FUSED) colblocks[k]++;
          }
    }
    if (serve) emit_prep(cols);
    // emit per fine column q = (kq, cq) in order: the chains into each block
    // of that column, then its final POTRF / TRSM.
    for (int kq = 0; kq < cols; ++kq) {
      L.structure(kq, st);
      std::vector<int> tiles_below;  // tiles i of column kq: kq itself, then struct(kq)
      tiles_below.push_back(kq);
      for (int i : st) tiles_below.push_back(i);
      for (int cq = 0; cq < L.nblk(kq); ++cq) {
        for (int i : tiles_below)
          for (int r = (i == kq ? cq : 0); r < L.nblk(i); ++r) emit_block_chain(i, r, kq, cq);
      }
    }
  }

  // Request server: one PREP task per tile column (the only roots).
  void emit_prep(int cols) {
    prep_ctr.resize(cols);
    const int64_t n = (int64_t)s.nt * s.b + s.a;
    for (int k = 0; k < cols; ++k) {
      prep_ctr[k] = newctr(false);
      Task t = blank(OP_PREP, 0, 0);
      const int64_t slot = L.tile(k, k);
      t.out = mkref(BUF_L, slot);
      t.cin = mkref(BUF_A, slot);
      const int64_t row0 = (int64_t)k * s.b;
      t.aux = mkref(BUF_A, L.doubles() + row0);
      t.ldo = s.b;
      t.ldc = s.a;
      t.ldx = L.nsub(k);
      t.zrows = s.w;
      t.diag = (int32_t)row0;
      t.gcol = (int32_t)n;
      if (k == s.nt) t.flags |= TF_CORNER;
      t.flags |= TF_URGENT * (k == 0);
      const double elems = k == s.nt ? (double)s.a * s.a : (double)(1 + L.nsub(k)) * s.b * s.b + (double)s.a * s.b;
      emit(t, {}, {}, {prep_ctr[k]}, elems * 0.02);
    }
  }

  // Source tile columns k < kq that update blocks (i, kq): kq and i both in
  // struct(k).
  void sources(int i, int kq, std::vector<int>& ks) {
    ks.clear();
    int k0 = kq - s.w;
    if (kq == s.nt) k0 = 0;  // the corner receives from every band column
    if (k0 < 0) k0 = 0;
    for (int k = k0; k < kq; ++k) {
      bool kq_in = (kq == s.nt) ? (s.a > 0) : (kq <= k + L.nsub(k));
      bool i_in = (i == s.nt) ? (s.a > 0) : (i <= k + L.nsub(k));
      if (kq_in && i_in) ks.push_back(k);
    }
  }

  // Global index of fine row block (i, r) (band tiles have nblk(0) blocks each).
  int64_t grow(int i, int r) const { return (int64_t)i * L.nblk(0) + r; }

  void emit_block_chain(int i, int r, int kq, int cq) {
    const int m = L.bdim(i, r), n = L.bdim(kq, cq);
    const bool diag = (i == kq && r == cq);
    // The factorization's critical path runs down the diagonal: POTRF(c) ->
    // TRSM(c+1, c) -> update of (c+1, c+1) from column c -> POTRF(c+1). Tasks
    // at the frontier are urgent (queued ahead of all others): every POTRF,
    // the TRSMs of the kUrgentReach blocks below a diagonal block, and the
    // updates from block column c into blocks whose row is within
    // kUrgentReach of c. Work further below has slack of one block step or
    // more and runs in list-schedule order, so the urgent queue stays short.
    constexpr int64_t kUrgentReach = 3;
    const int64_t dist = grow(i, r) - grow(kq, cq);
    const int32_t me = lctr[lidx(i, kq, r, cq)];
    // terms: list of (source tile column k, first block c0, last block c1)
    struct Term { int k, c0, c1; };
    std::vector<Term> terms;
    std::vector<int> ks;
    sources(i, kq, ks);
    // Updates from tile columns older than kq-1 were final long before this
    // block is due: batch them (kChunkOld block columns per task). Updates from
    // tile column kq-1 and from kq itself arrive one block column at a time
    // along the critical path: one block column per task.
    const int kChunkOld = tune_chunk_old(s.tune);
    for (int k : ks) {
      const int step = (k < kq - 1) ? kChunkOld : 1;
      for (int c0 = 0; c0 < L.nblk(k); c0 += step) terms.push_back({k, c0, std::min(L.nblk(k), c0 + step) - 1});
    }
    for (int c = 0; c < cq; ++c) terms.push_back({kq, c, c});  // same tile column: one block column per task
    // A block of block column cq is due when the factorization frontier
    // reaches that column. Its one-block-column terms whose source lies more
    // than kFuseReach block columns before cq are final long before that:
    // merge runs of them (one source tile column per run) into one task of up
    // to kFuseCols block columns (a longer inner length: the epilogue,
    // completion and, in the emulated modes, the recombination are paid once
    // per run instead of once per column). The nearer terms, which arrive one
    // frontier step at a time, and the block's newest term stay single.
    // A run lumps the work of a block's chain, which lengthens the factor's
    // critical path: it pays only when the whole selected inversion runs in
    // the same launch and keeps the GPU busy meanwhile (a fused plan of every
    // column), not in a factor-only or column-selected plan, whose time is
    // the factor's critical path.
    constexpr int64_t kFuseReach = 8;
    const int kFuseCols = kind == PLAN_FUSED && s.sel0 == 0 ? 8 : 1;
    {
      std::vector<Term> merged;
      for (size_t q = 0; q < terms.size(); ++q) {
        const Term& t = terms[q];
        if (!merged.empty() && q + 1 < terms.size()) {
          Term& p = merged.back();
          if (p.k == t.k && t.c0 == t.c1 && p.c1 + 1 == t.c0 && t.c1 - p.c0 < kFuseCols &&
              grow(kq, cq) - grow(t.k, t.c1) > kFuseReach) {
            p.c1 = t.c1;
            continue;
          }
        }
        merged.push_back(t);
      }
      terms.swap(merged);
    }
    const int64_t outref = mkref(BUF_L, L.blk(i, kq, r, cq));
    const int ld_i = L.rows(i);
    int nwritten = 0;
    auto term_seg = [&](const Term& t) {
      int64_t a = mkref(BUF_L, L.blk(i, t.k, r, t.c0));
      int64_t b = mkref(BUF_L, L.blk(kq, t.k, cq, t.c0));
      int kk = std::min(L.rows(t.k), (t.c1 + 1) * FB) - t.c0 * FB;
      return seg(a, ld_i, b, L.rows(kq), kk, false, true);
    };
    auto term_waits = [&](const Term& t, std::vector<Wait>& w) {
      w.push_back({lctr[lidx(i, t.k, r, t.c1)], lfinal[lidx(i, t.k, r, t.c1)]});
      w.push_back({lctr[lidx(kq, t.k, cq, t.c1)], lfinal[lidx(kq, t.k, cq, t.c1)]});
    };
    const size_t nfused = 0;  // every update runs as its own (split) task
    size_t nchain = terms.size() - nfused;
    // The critical path's links run as small parts on more CTAs: the FP64
    // newest update of a diagonal block as three quadrant tasks of 16 x 16
    // parts, the final TRSM of the block right below a diagonal block as two
    // tasks of 8-row parts (they write disjoint parts of the block)
    const bool newest_fp64 = nchain > 0 && (s.prec == PREC_FP64 ||
                                            (i == kq && terms[nchain - 1].k == kq && !tune_lower_diag(s.tune)));
    const bool fine_newest = diag && m == n && m > 32 && newest_fp64;
    const bool fine_final = !diag && dist == 1 && m > 32;
    // writers of the block's chain counter `me` (strictly ordered); the
    // quadrant tasks and the two final TRSM halves run side by side and
    // signal counters of their own
    int total_writers = (int)nchain + 1 - (fine_newest ? 1 : 0);
    lfinal[lidx(i, kq, r, cq)] = total_writers;
    bool written = false;  // the block already holds an update (read it from L, not A)
    int32_t qctr = -1;     // the quadrant tasks of the newest update
    for (size_t t = 0; t < nchain; ++t) {
      if (fine_newest && t + 1 == nchain) {
        const Seg sg = term_seg(terms[t]);
        const int qr[3] = {0, 32, 32}, qc[3] = {0, 0, 32};
        qctr = newctr(false);
        for (int x = 0; x < 3; ++x) {
          const int64_t off = qr[x] + (int64_t)qc[x] * ld_i;
          Task tq = blank(OP_UPD, std::min(32, m - qr[x]), std::min(32, n - qc[x]));
          tq.out = outref + off;
          tq.ldo = ld_i;
          tq.cin = (written ? outref : mkref(BUF_A, L.blk(i, kq, r, cq))) + off;
          tq.ldc = ld_i;
          split(tq, x == 1 ? PM_QUAD16 : PM_TRI16);
          if (grow(i, r) - grow(terms[t].k, terms[t].c1) <= kUrgentReach) tq.flags |= TF_URGENT;
          Seg sq = sg;
          sq.a += qr[x];
          sq.b += qc[x];
          std::vector<Wait> w;
          if (nwritten > 0) w.push_back({me, nwritten});
          if (!written && serve) w.push_back({prep_ctr[kq], 1});
          term_waits(terms[t], w);
          emit(tq, {sq}, w, {qctr}, 0.0);
        }
        written = true;
        continue;
      }
      Task tk = blank(OP_UPD, m, n);
      tk.out = outref;
      tk.ldo = ld_i;
      tk.cin = written ? outref : mkref(BUF_A, L.blk(i, kq, r, cq));
      tk.ldc = ld_i;
      // a diagonal block only needs its lower quadrants; the newest update of
      // a block gates its TRSM / POTRF on the critical path: split it 4 ways
      if (diag) split(tk, PM_TRI3);
      else if (t + 1 == nchain && tune_upd_split(s.tune) == 0) split(tk, PM_QUAD4);
      if (grow(i, r) - grow(terms[t].k, terms[t].c1) <= kUrgentReach) tk.flags |= TF_URGENT;
      // the diagonal tile's own updates belong to its POTRF, which stays true
      // FP64 unless the tuning code lowers them too
      if (!(i == kq && terms[t].k == kq) || tune_lower_diag(s.tune)) lower_precision(tk);
      std::vector<Wait> w;
      if (nwritten > 0) w.push_back({me, nwritten});
      if (!written && serve) w.push_back({prep_ctr[kq], 1});
      term_waits(terms[t], w);
      sym_block = diag;
      emit(tk, {term_seg(terms[t])}, w, {me}, 0.0);
      ++nwritten;
      written = true;
    }
    // final task
    std::vector<Seg> segs;
    std::vector<Wait> w;
    if (nwritten > 0) w.push_back({me, nwritten});
    if (qctr >= 0) w.push_back({qctr, 3});
    if (!written && serve) w.push_back({prep_ctr[kq], 1});
    for (size_t t = nchain; t < terms.size(); ++t) {
      segs.push_back(term_seg(terms[t]));
      term_waits(terms[t], w);
    }
    if (fine_final) {
      // the two halves signal a counter of their own, which replaces the
      // block's chain counter for every later reader (both are predecessors)
      const int32_t dctr = lctr[lidx(kq, kq, cq, cq)];
      w.push_back({dctr, lfinal[lidx(kq, kq, cq, cq)]});
      const int32_t fctr = newctr(false);
      if (kind == PLAN_FUSED) colblocks[kq]++;  // two final tasks signal the column
      for (int h = 0; h < 2; ++h) {
        const int r0 = 32 * h;
        Task tq = blank(OP_TRSM_RLT, std::min(32, m - r0), n);
        split(tq, PM_ROWS8);
        tq.flags |= TF_URGENT;
        tq.out = outref + r0;
        tq.ldo = ld_i;
        tq.cin = (written ? outref : mkref(BUF_A, L.blk(i, kq, r, cq))) + r0;
        tq.ldc = ld_i;
        tq.aux = mkref(BUF_L, L.blk(kq, kq, cq, cq));
        tq.ldx = L.rows(kq);
        std::vector<Seg> sh = segs;
        for (Seg& g : sh) g.a += r0;
        std::vector<int32_t> sig{fctr};
        if (kind == PLAN_FUSED) sig.push_back(colfinal[kq]);
        emit(tq, sh, w, sig, 2.0 * n * kSweepStepNs);
      }
      lctr[lidx(i, kq, r, cq)] = fctr;
      lfinal[lidx(i, kq, r, cq)] = 2;
      return;
    }
    Task tk = blank(diag ? OP_POTRF : OP_TRSM_RLT, m, n);
    if (!diag) split(tk, PM_ROWS4);
    if (diag || dist <= kUrgentReach) tk.flags |= TF_URGENT;
    tk.out = outref;
    tk.ldo = ld_i;
    tk.cin = written ? outref : mkref(BUF_A, L.blk(i, kq, r, cq));
    tk.ldc = ld_i;
    std::vector<int32_t> sig{me};
    double epi;
    if (diag) {
      tk.diag = ndiag++;
      tk.gcol = kq * s.b + cq * FB;
      epi = 3.0 * m * kSweepStepNs;
    } else {
      const int32_t dctr = lctr[lidx(kq, kq, cq, cq)];
      w.push_back({dctr, lfinal[lidx(kq, kq, cq, cq)]});
      tk.aux = mkref(BUF_L, L.blk(kq, kq, cq, cq));
      tk.ldx = L.rows(kq);
      epi = 2.0 * n * kSweepStepNs;
    }
    if (kind == PLAN_FUSED) sig.push_back(colfinal[kq]);
    emit(tk, segs, w, sig, epi);
    if (diag && cq > 0) {
      // L's strict upper part in this block column of the diagonal tile: no
      // task reads it, so it is written by a task of its own, off the
      // critical path (after the request's A in a served launch, which
      // builds A in place in L)
      Task z = blank(OP_ZERO, m, n);
      z.out = outref;
      z.ldo = ld_i;
      z.zrows = cq * FB;
      std::vector<Wait> zw;
      if (serve) zw.push_back({prep_ctr[kq], 1});
      emit(z, {}, zw, {}, 0.08 * z.zrows * n);
    }
  }

  // ------------------------------------------------------------ selinv ----
  // Counters: Linv column panels (chain), Sigma^0 blocks (chain), U column
  // panels, Sigma row / column panels (diagonal tiles: lower blocks only).
  std::vector<int32_t> linv_col;   // [i][c]
  std::vector<int64_t> linv_base;
  std::vector<int32_t> s0_ctr;     // [i][r][c] lower
  std::vector<int64_t> s0_base;
  std::vector<int32_t> u_col;      // per (k,i) tile: column panels
  std::vector<int32_t> s_row, s_col;  // per Sigma tile: row / column panels
  std::vector<int64_t> ut_base, st_rbase, st_cbase;  // indexed by tile slot like lctr_base

  int64_t slot_index(int i, int k) const { return (int64_t)k * (s.w + 2) + tile_slot(i, k); }

  void build_selinv() {
    const int cols = L.last() + 1;
    std::vector<int> st;
    linv_base.assign(cols, 0);
    s0_base.assign(cols, 0);
    ut_base.assign((size_t)cols * (s.w + 2), -1);
    st_rbase.assign((size_t)cols * (s.w + 2), -1);
    st_cbase.assign((size_t)cols * (s.w + 2), -1);
    for (int i = 0; i < cols; ++i) {
      const int R = L.nblk(i);
      linv_base[i] = linv_col.size();
      for (int c = 0; c < R; ++c) linv_col.push_back(newctr(true));
      s0_base[i] = s0_ctr.size();
      for (int r = 0; r < R; ++r)
        for (int c = 0; c <= r; ++c) s0_ctr.push_back(newctr(true));
      // Sigma diag tile panels
      st_rbase[slot_index(i, i)] = s_row.size();
      for (int r = 0; r < R; ++r) s_row.push_back(newctr(false));
      st_cbase[slot_index(i, i)] = s_col.size();
      for (int c = 0; c < R; ++c) s_col.push_back(newctr(false));
      L.structure(i, st);
      for (int k : st) {
        ut_base[slot_index(k, i)] = u_col.size();
        for (int c = 0; c < R; ++c) u_col.push_back(newctr(false));
        st_rbase[slot_index(k, i)] = s_row.size();
        for (int r = 0; r < L.nblk(k); ++r) s_row.push_back(newctr(false));
        st_cbase[slot_index(k, i)] = s_col.size();
        for (int c = 0; c < R; ++c) s_col.push_back(newctr(false));
      }
    }
    // Sigma of tile column i depends only on Sigma of the columns after it and
    // on column i's own phase 1: a selection starting at column sel0 needs
    // exactly the phase-1 and phase-2 work of columns >= sel0.
    if (kind == PLAN_FUSED) {
      // one join per tile column waits for all of its L blocks; the column's
      // phase-1 tasks wait for the join (one dependency each instead of one
      // per L block: a column of ~400 blocks and ~400 phase-1 tasks)
      coljoin.assign(cols, -1);
      for (int i = s.sel0; i < cols; ++i) {
        coljoin[i] = newctr(true);
        emit(blank(OP_JOIN, 0, 0), {}, {{colfinal[i], colblocks[i]}}, {coljoin[i]}, 0.0);
      }
    }
    for (int i = s.sel0; i < cols; ++i) emit_phase1(i);
    for (int i = cols - 1; i >= s.sel0; --i) emit_phase2(i);
  }

  int32_t linv_ctr(int i, int c) const { return linv_col[linv_base[i] + c]; }
  int32_t s0(int i, int r, int c) const { return s0_ctr[s0_base[i] + (int64_t)r * (r + 1) / 2 + c]; }
  int32_t ucol(int k, int i, int c) const { return u_col[ut_base[slot_index(k, i)] + c]; }
  int32_t srow(int j, int i, int r) const { return s_row[st_rbase[slot_index(j, i)] + r]; }
  int32_t scol(int j, int i, int c) const { return s_col[st_cbase[slot_index(j, i)] + c]; }

  void add_fused_wait(int i, std::vector<Wait>& w) {
    if (kind == PLAN_FUSED) w.push_back({coljoin[i], 1});
  }

  void emit_phase1(int i) {
    const int R = L.nblk(i), ld = L.rows(i);
    std::vector<int> st;
    // TRTRI of the diagonal tile, block column by block column
    for (int c = 0; c < R; ++c) {
      for (int r = c; r < R; ++r) {
        const int m = L.bdim(i, r), n = L.bdim(i, c);
        std::vector<Wait> w;
        add_fused_wait(i, w);
        if (r == c) {
          Task t = blank(OP_TRTRI, m, n);
          t.out = mkref(BUF_W, L.blk(i, i, r, c));
          t.ldo = ld;
          t.aux = mkref(BUF_L, L.blk(i, i, r, r));
          t.ldx = ld;
          emit(t, {}, w, {linv_ctr(i, c)}, 2.0 * m * kSweepStepNs);
        } else {
          // Linv[r,c] = -L[r,r]^{-1} sum_{q=c}^{r-1} L[r,q] Linv[q,c]
          Task t = blank(OP_TRSM_LLN, m, n);
          t.out = mkref(BUF_W, L.blk(i, i, r, c));
          t.ldo = ld;
          t.aux = mkref(BUF_L, L.blk(i, i, r, r));
          t.ldx = ld;
          w.push_back({linv_ctr(i, c), r - c});
          Seg g = seg(mkref(BUF_L, L.blk(i, i, r, c)), ld, mkref(BUF_W, L.blk(i, i, c, c)), ld, (r - c) * FB, false,
                      false);
          emit(t, {g}, w, {linv_ctr(i, c)}, 2.0 * m * kSweepStepNs);
        }
      }
    }
    // LAUUM: Sigma^0[r,c] = sum_{q>=r} Linv[q,r]^T Linv[q,c], r >= c
    for (int r = 0; r < R; ++r)
      for (int c = 0; c <= r; ++c) {
        const int m = L.bdim(i, r), n = L.bdim(i, c);
        Task t = blank(OP_STORE, m, n);
        if (r == c) split(t, PM_TRI3);  // only the lower part of a diagonal block is used
        t.out = mkref(BUF_S, L.blk(i, i, r, c));
        t.ldo = ld;
        std::vector<Wait> w{{linv_ctr(i, r), R - r}, {linv_ctr(i, c), R - c}};
        Seg g = seg(mkref(BUF_W, L.blk(i, i, r, r)), ld, mkref(BUF_W, L.blk(i, i, r, c)), ld, ld - r * FB, true,
                    false);
        emit(t, {g}, w, {s0(i, r, c)}, 0.0);
      }
    // TRMM: U_ki = L_ki Linv_ii
    L.structure(i, st);
    for (int k : st) {
      const int ldk = L.rows(k);
      for (int c = 0; c < R; ++c)
        for (int r = 0; r < L.nblk(k); ++r) {
          const int m = L.bdim(k, r), n = L.bdim(i, c);
          Task t = blank(OP_STORE, m, n);
          t.out = mkref(BUF_W, L.blk(k, i, r, c));
          t.ldo = ldk;
          std::vector<Wait> w;
          add_fused_wait(i, w);
          w.push_back({linv_ctr(i, c), R - c});
          Seg g = seg(mkref(BUF_L, L.blk(k, i, r, c)), ldk, mkref(BUF_W, L.blk(i, i, c, c)), ld, ld - c * FB, false,
                      false);
          lower_precision(t);
          emit(t, {g}, w, {ucol(k, i, c)}, 0.0);
        }
    }
  }

  void emit_phase2(int i) {
    const int R = L.nblk(i), ld = L.rows(i);
    std::vector<int> st;
    L.structure(i, st);
    // off-diagonal tiles, j from the last down (Algorithm 3's j loop)
    for (int tj = (int)st.size() - 1; tj >= 0; --tj) {
      const int j = st[tj], ldj = L.rows(j);
      for (int c = 0; c < R; ++c)
        for (int r = 0; r < L.nblk(j); ++r) {
          const int m = L.bdim(j, r), n = L.bdim(i, c);
          Task t = blank(OP_NEG, m, n);
          split_p2(t);  // phase 2 is a chain of joins: shorter tasks, shorter steps
          t.out = mkref(BUF_S, L.blk(j, i, r, c));
          t.ldo = ldj;
          std::vector<Seg> segs;
          std::vector<Wait> w;
          for (int k : st) {
            const int ldk = L.rows(k);
            if (j == k) {
              segs.push_back(seg(mkref(BUF_S, L.blk(j, j, r, 0)), ldj, mkref(BUF_W, L.blk(k, i, 0, c)), ldk, ldk,
                                 false, false));
              w.push_back({srow(j, j, r), r + 1});
              w.push_back({scol(j, j, r), L.nblk(j) - r});
            } else if (j > k) {
              segs.push_back(seg(mkref(BUF_S, L.blk(j, k, r, 0)), ldj, mkref(BUF_W, L.blk(k, i, 0, c)), ldk, ldk,
                                 false, false));
              w.push_back({srow(j, k, r), L.nblk(k)});
            } else {
              segs.push_back(seg(mkref(BUF_S, L.blk(k, j, 0, r)), ldk, mkref(BUF_W, L.blk(k, i, 0, c)), ldk, ldk,
                                 true, false));
              w.push_back({scol(k, j, r), L.nblk(k)});
            }
            w.push_back({ucol(k, i, c), L.nblk(k)});
          }
          lower_precision(t);
          emit(t, segs, w, {srow(j, i, r), scol(j, i, c)}, 0.0);
        }
      tile_gemms += (long long)st.size();
    }
    // diagonal tile: Sigma_ii = Sigma^0 - sum_k Sigma_ki^T U_ki (lower blocks, mirrored)
    for (int r = 0; r < R; ++r)
      for (int c = 0; c <= r; ++c) {
        const int m = L.bdim(i, r), n = L.bdim(i, c);
        Task t = blank(OP_SYMUPD, m, n);
        if (r == c) split(t, PM_TRI3);
        else split_p2(t);
        t.out = mkref(BUF_S, L.blk(i, i, r, c));
        t.ldo = ld;
        t.cin = t.out;
        t.ldc = ld;
        if (r != c) {
          t.aux = mkref(BUF_S, L.blk(i, i, c, r));
          t.ldx = ld;
        } else {
          t.flags = TF_SYM_DIAG;
        }
        std::vector<Seg> segs;
        std::vector<Wait> w{{s0(i, r, c), 1}};
        for (int k : st) {
          const int ldk = L.rows(k);
          segs.push_back(seg(mkref(BUF_S, L.blk(k, i, 0, r)), ldk, mkref(BUF_W, L.blk(k, i, 0, c)), ldk, ldk, true,
                             false));
          w.push_back({scol(k, i, r), L.nblk(k)});
          w.push_back({ucol(k, i, c), L.nblk(k)});
        }
        if (!segs.empty()) lower_precision(t);  // the products; the assembly (cin - acc, mirror) stays FP64
        sym_block = r == c;
        emit(t, segs, w, {srow(i, i, r), scol(i, i, c)}, 0.0);
      }
    tile_gemms += (long long)st.size();
  }

  // ---------------------------------------------------------- schedule ----
  int finish(int workers) {
    const int nt_ = (int)tasks.size();
    // predecessor edges from waits (flat, per task sorted and unique); the
    // emission order must be topological
    // writers of each counter, in emission order
    const int64_t nctr = (int64_t)chain.size();
    std::vector<int64_t> woff(nctr + 1, 0);
    for (int32_t c : fsigs) {
      if (c < 0 || c >= nctr) return STILES_ERR_PLAN;
      woff[c + 1]++;
    }
    for (int64_t c = 0; c < nctr; ++c) woff[c + 1] += woff[c];
    std::vector<int32_t> wr(fsigs.size());
    {
      std::vector<int64_t> fill(woff.begin(), woff.end() - 1);
      for (int t = 0; t < nt_; ++t)
        for (int64_t e = sig_off[t]; e < sig_off[t + 1]; ++e) wr[fill[fsigs[e]]++] = t;
    }
    std::vector<int64_t> poff(nt_ + 1, 0);
    std::vector<int32_t> pred;
    pred.reserve(fwaits.size() + fwaits.size() / 2);
    std::vector<int32_t> scratch;
    for (int t = 0; t < nt_; ++t) {
      scratch.clear();
      for (int64_t e = wait_off[t]; e < wait_off[t + 1]; ++e) {
        const Wait& w = fwaits[e];
        if (w.ctr < 0 || w.ctr >= nctr) return STILES_ERR_PLAN;
        const int64_t w0 = woff[w.ctr], nw = woff[w.ctr + 1] - w0;
        if (w.need > nw || w.need < 0) return STILES_ERR_PLAN;
        if (w.need == 0) continue;
        if (chain[w.ctr]) scratch.push_back(wr[w0 + w.need - 1]);
        else scratch.insert(scratch.end(), wr.begin() + w0, wr.begin() + w0 + w.need);
      }
      std::sort(scratch.begin(), scratch.end());
      scratch.erase(std::unique(scratch.begin(), scratch.end()), scratch.end());
      if (!scratch.empty() && scratch.back() >= t) return STILES_ERR_PLAN;
      pred.insert(pred.end(), scratch.begin(), scratch.end());
      poff[t + 1] = (int64_t)pred.size();
    }
    if (pred.size() > (size_t)INT32_MAX) return STILES_ERR_PLAN;
    // successors of each task, in ascending task order
    std::vector<int64_t> soff(nt_ + 1, 0);
    for (int32_t q : pred) soff[q + 1]++;
    for (int t = 0; t < nt_; ++t) soff[t + 1] += soff[t];
    std::vector<int32_t> succ(pred.size());
    std::vector<int32_t> indeg(nt_, 0);
    {
      std::vector<int64_t> fill(soff.begin(), soff.end() - 1);
      for (int t = 0; t < nt_; ++t) {
        indeg[t] = (int32_t)(poff[t + 1] - poff[t]);
        for (int64_t e = poff[t]; e < poff[t + 1]; ++e) succ[fill[pred[e]]++] = t;
      }
    }
    std::vector<int32_t>().swap(pred);
    std::vector<int64_t>().swap(poff);
    std::vector<int32_t>().swap(wr);
    std::vector<int64_t>().swap(woff);
    // bottom levels
    std::vector<double> blevel(nt_, 0.0);
    double cp = 0;
    for (int t = nt_ - 1; t >= 0; --t) {
      double best = 0;
      for (int64_t e = soff[t]; e < soff[t + 1]; ++e) best = std::max(best, blevel[succ[e]]);
      blevel[t] = cost[t] + best;
      cp = std::max(cp, blevel[t]);
    }
    // list schedule: free workers take the ready task with the largest bottom level
    using RItem = std::pair<double, int32_t>;
    using EItem = std::pair<double, int32_t>;  // (finish time, task)
    std::vector<RItem> rbuf;
    rbuf.reserve(nt_);
    std::priority_queue<RItem> ready(std::less<RItem>(), std::move(rbuf));
    std::vector<EItem> ebuf;
    ebuf.reserve((size_t)std::max(1, workers) + 1);
    std::priority_queue<EItem, std::vector<EItem>, std::greater<EItem>> running(std::greater<EItem>(), std::move(ebuf));
    for (int t = 0; t < nt_; ++t)
      if (indeg[t] == 0) ready.push({blevel[t], t});
    std::vector<int32_t> order;
    order.reserve(nt_);
    double now = 0;
    int free_workers = std::max(1, workers);
    auto release = [&](int32_t t) {
      for (int64_t e = soff[t]; e < soff[t + 1]; ++e)
        if (--indeg[succ[e]] == 0) ready.push({blevel[succ[e]], succ[e]});
    };
    while ((int)order.size() < nt_) {
      while (free_workers > 0 && !ready.empty()) {
        int32_t t = ready.top().second;
        ready.pop();
        order.push_back(t);
        running.push({now + cost[t], t});
        --free_workers;
      }
      if (running.empty()) return STILES_ERR_PLAN;  // cycle
      EItem e = running.top();
      running.pop();
      now = e.first;
      ++free_workers;
      release(e.second);
      while (!running.empty() && running.top().first <= now) {
        EItem e2 = running.top();
        running.pop();
        ++free_workers;
        release(e2.second);
      }
    }
    while (!running.empty()) { now = std::max(now, running.top().first); running.pop(); }
    // write the plan in list-schedule order (the device queue order)
    Plan& p = *out;
    p.tasks.clear(); p.segs.clear(); p.waits.clear(); p.sigs.clear();
    p.tasks.reserve(nt_); p.segs.reserve(fsegs.size()); p.waits.reserve(fwaits.size()); p.sigs.reserve(fsigs.size());
    std::vector<int32_t> rank(nt_);
    for (int r = 0; r < nt_; ++r) rank[order[r]] = r;
    for (int32_t t : order) {
      Task tk = tasks[t];
      tk.seg0 = (int32_t)p.segs.size();
      tk.nseg = (int32_t)(seg_off[t + 1] - seg_off[t]);
      p.segs.insert(p.segs.end(), fsegs.begin() + seg_off[t], fsegs.begin() + seg_off[t + 1]);
      tk.wait0 = (int32_t)p.waits.size();
      tk.nwait = (int32_t)(wait_off[t + 1] - wait_off[t]);
      p.waits.insert(p.waits.end(), fwaits.begin() + wait_off[t], fwaits.begin() + wait_off[t + 1]);
      tk.sig0 = (int32_t)p.sigs.size();
      tk.nsig = (int16_t)(sig_off[t + 1] - sig_off[t]);
      p.sigs.insert(p.sigs.end(), fsigs.begin() + sig_off[t], fsigs.begin() + sig_off[t + 1]);
      p.tasks.push_back(tk);
    }
    // successor graph in schedule-order indices
    p.indeg.assign(nt_, 0);
    p.succ_off.assign(nt_ + 1, 0);
    p.succ.clear();
    p.succ.reserve(succ.size());
    for (int r = 0; r < nt_; ++r) {
      const int32_t t = order[r];
      p.succ_off[r] = (int32_t)p.succ.size();
      for (int64_t e = soff[t]; e < soff[t + 1]; ++e) {
        p.succ.push_back(rank[succ[e]]);
        p.indeg[rank[succ[e]]]++;
      }
    }
    p.succ_off[nt_] = (int32_t)p.succ.size();
    p.nbuckets = (nt_ + kTasksPerBucket - 1) / kTasksPerBucket;
    p.slots0.assign((size_t)p.nbuckets * kSlotsPerBucket, -1);
    p.tail0.assign(p.nbuckets, 0);
    p.bcap.assign(p.nbuckets, 0);
    p.urgent_parts = 0;
    p.urgent_tail0 = 0;
    for (int r = 0; r < nt_; ++r) {
      const int parts = p.tasks[r].parts;
      if (p.tasks[r].flags & TF_URGENT) {
        p.urgent_parts += parts;
        continue;
      }
      const int b = r / kTasksPerBucket;
      p.bcap[b] += parts;
      if (p.indeg[r] == 0)
        for (int q = 0; q < parts; ++q) p.slots0[(size_t)b * kSlotsPerBucket + p.tail0[b]++] = 4 * r + q;
    }
    p.uslots0.assign(std::max(1, p.urgent_parts), -1);
    for (int r = 0; r < nt_; ++r)
      if ((p.tasks[r].flags & TF_URGENT) && p.indeg[r] == 0)
        for (int q = 0; q < p.tasks[r].parts; ++q) p.uslots0[p.urgent_tail0++] = 4 * r + q;
    p.nctr = (int32_t)chain.size();
    p.ndiag = ndiag;
    p.flops = flops;
    p.flops_lowered = flops_lowered;
    p.tile_gemms = tile_gemms;
    p.cp_ns = cp;
    p.makespan_ns = now;
    return 0;
  }
};

}  // namespace

// Algorithmic flops of the tile operations (the counting convention used for
// every TFLOP/s figure): POTRF, TRTRI, LAUUM m^3/3; TRSM, TRMM m k^2;
// SYRK m^2 k; GEMM 2 m n k; the symmetric Sigma_ii update m^2 k per term
// (only its lower triangle is computed, like SYRK).
double tile_flops(const Shape& s, PlanKind kind) {
  Layout L(s);
  std::vector<int> st;
  double f = 0;
  const int cols = L.last() + 1;
  for (int k = 0; k < cols; ++k) {
    const double mk = L.rows(k);
    L.structure(k, st);
    if (kind != PLAN_SELINV) {
      f += mk * mk * mk / 3.0;                          // POTRF
      for (size_t t = 0; t < st.size(); ++t) {
        const double mi = L.rows(st[t]);
        f += mi * mk * mk;                              // TRSM
        f += mi * mi * mk;                              // SYRK
        for (size_t u = 0; u < t; ++u) f += 2.0 * mi * L.rows(st[u]) * mk;  // GEMM
      }
    }
    if (kind != PLAN_FACTOR && k >= s.sel0) {
      f += 2.0 * mk * mk * mk / 3.0;                    // TRTRI + LAUUM
      for (int j : st) {
        const double mj = L.rows(j);
        f += mj * mk * mk;                              // TRMM
        for (int q : st) f += 2.0 * mj * mk * L.rows(q);  // Sigma_jk U_ki
        f += mk * mk * mj;                              // Sigma_kk update
      }
    }
  }
  return f;
}

// Task-table size estimate: about (1+w+1) tiles per column, nblk^2 blocks per
// tile and up to (w+1)*nblk + nblk chain tasks per block.
static double task_estimate(const Shape& s) {
  const double nb = (s.b + FB - 1) / FB, na = (s.a + FB - 1) / FB;
  return (double)s.nt * (s.w + 2) * nb * (nb + na) * ((s.w + 2) * nb + 8);
}

static bool shape_ok(const Shape& s) {
  return s.nt >= 1 && s.b >= 1 && s.w >= 0 && s.a >= 0 && s.w <= s.nt - 1 && tune_valid(s.tune) && s.sel0 >= 0 &&
         s.sel0 <= (s.a > 0 ? s.nt : s.nt - 1);
}

int build_plan(const Shape& s, PlanKind kind, int workers, Plan* out) {
  if (!shape_ok(s)) return STILES_ERR_INVALID_ARG;
  if (task_estimate(s) > 4.0e8) return STILES_ERR_INVALID_ARG;
  Builder B(s, kind, out);
  if (kind == PLAN_FACTOR || kind == PLAN_FUSED) B.build_factor();
  if (kind == PLAN_SELINV || kind == PLAN_FUSED) B.build_selinv();
  B.flops = tile_flops(s, kind);
  int rc = B.finish(workers);
  if (rc) return rc;
  return check_plan(*out);
}

int build_serve_template(const Shape& s, int workers, Plan* out) {
  if (!shape_ok(s)) return STILES_ERR_INVALID_ARG;
  if (task_estimate(s) > 4.0e8) return STILES_ERR_INVALID_ARG;
  Builder B(s, PLAN_FUSED, out);
  B.serve = true;
  B.build_factor();
  B.build_selinv();
  B.flops = tile_flops(s, PLAN_FUSED);
  int rc = B.finish(workers);
  if (rc) return rc;
  return check_plan(*out);
}

int build_batch_plan(const std::vector<Shape>& shapes, const std::vector<int64_t>& base, int workers, Plan* out,
                     std::vector<int32_t>* diag_base) {
  if (shapes.empty() || base.size() != shapes.size() || !out || !diag_base) return STILES_ERR_INVALID_ARG;
  double est = 0;
  for (const Shape& s : shapes) {
    if (!shape_ok(s) || s.prec != shapes[0].prec) return STILES_ERR_INVALID_ARG;
    est += task_estimate(s);
  }
  if (est > 4.0e8) return STILES_ERR_INVALID_ARG;
  Builder M(shapes[0], PLAN_FUSED, out);
  diag_base->assign(shapes.size() + 1, 0);
  for (size_t m = 0; m < shapes.size(); ++m) {
    Builder B(shapes[m], PLAN_FUSED, nullptr);
    B.build_factor();
    B.build_selinv();
    const int32_t coff = (int32_t)M.chain.size(), doff = M.ndiag;
    const int64_t off = base[m];
    auto shift = [off](int64_t ref) { return ref < 0 ? ref : ref + off; };
    for (size_t t = 0; t < B.tasks.size(); ++t) {
      Task tk = B.tasks[t];
      tk.out = shift(tk.out);
      tk.cin = shift(tk.cin);
      tk.aux = shift(tk.aux);
      if (tk.diag >= 0) tk.diag += doff;
      M.tasks.push_back(tk);
    }
    M.cost.insert(M.cost.end(), B.cost.begin(), B.cost.end());
    for (Seg g : B.fsegs) {
      g.a = shift(g.a);
      g.b = shift(g.b);
      M.fsegs.push_back(g);
    }
    for (Wait w : B.fwaits) {
      w.ctr += coff;
      M.fwaits.push_back(w);
    }
    for (int32_t c : B.fsigs) M.fsigs.push_back(c + coff);
    for (size_t t = 0; t < B.tasks.size(); ++t) {
      M.seg_off.push_back(M.seg_off.back() + (B.seg_off[t + 1] - B.seg_off[t]));
      M.wait_off.push_back(M.wait_off.back() + (B.wait_off[t + 1] - B.wait_off[t]));
      M.sig_off.push_back(M.sig_off.back() + (B.sig_off[t + 1] - B.sig_off[t]));
    }
    M.chain.insert(M.chain.end(), B.chain.begin(), B.chain.end());
    M.ndiag += B.ndiag;
    M.tile_gemms += B.tile_gemms;
    M.flops += tile_flops(shapes[m], PLAN_FUSED);
    M.flops_lowered += B.flops_lowered;
    (*diag_base)[m + 1] = M.ndiag;
  }
  const int rc = M.finish(workers);
  if (rc) return rc;
  return check_plan(*out);
}

int check_plan(const Plan& p) {
  const int64_t ntasks = (int64_t)p.tasks.size();
  std::vector<int32_t> seen(p.nctr, 0);  // signals issued by tasks before the current one
  for (int64_t t = 0; t < ntasks; ++t) {
    const Task& tk = p.tasks[t];
    if (tk.wait0 < 0 || tk.nwait < 0 || (int64_t)tk.wait0 + tk.nwait > (int64_t)p.waits.size()) return STILES_ERR_PLAN;
    if (tk.seg0 < 0 || tk.nseg < 0 || (int64_t)tk.seg0 + tk.nseg > (int64_t)p.segs.size()) return STILES_ERR_PLAN;
    if (tk.sig0 < 0 || tk.nsig < 0 || (int64_t)tk.sig0 + tk.nsig > (int64_t)p.sigs.size()) return STILES_ERR_PLAN;
    if (tk.m < 0 || tk.n < 0 || tk.m > FB || tk.n > FB || tk.op > OP_JOIN) return STILES_ERR_PLAN;
    if (tk.parts < 1 || tk.parts > 4 || tk.pmode > PM_QUAD16 || tk.prec > PREC_FP32X) return STILES_ERR_PLAN;
    for (int q = 0; q < tk.nwait; ++q) {
      const Wait& w = p.waits[tk.wait0 + q];
      if (w.ctr < 0 || w.ctr >= p.nctr) return STILES_ERR_PLAN;
      if (w.need > seen[w.ctr]) return STILES_ERR_PLAN;  // would wait for a later task: can deadlock
    }
    for (int q = 0; q < tk.nsig; ++q) {
      int32_t c = p.sigs[tk.sig0 + q];
      if (c < 0 || c >= p.nctr) return STILES_ERR_PLAN;
      seen[c]++;
    }
  }
  return 0;
}

}  // namespace stiles

namespace stiles {

// Host emulation of one launch, for tests: every access of every task part
// stays inside its buffer (A, L, Sigma, scratch tiles: `doubles` each), every
// queue slot index stays inside its bucket or the urgent queue, and the
// successor graph releases every task exactly once. Returns 0 or
// STILES_ERR_PLAN (and prints the first problem to stderr).
int validate_plan(const Plan& p, const Shape& s, int kind) { return validate_plan_len(p, Layout(s).doubles(), kind); }

int validate_plan_len(const Plan& p, int64_t lim, int kind) {
  // buffers a launch of this kind provides: factor A, L, scratch; selinv L, Sigma, scratch
  const unsigned allowed = kind == PLAN_FACTOR ? 0xBu : kind == PLAN_SELINV ? 0xEu : 0xFu;
  const int nt = (int)p.tasks.size();
  auto bad = [&](const char* what, int t) {
    fprintf(stderr, "validate_plan: %s (task %d, op %d)\n", what, t, t >= 0 ? (int)p.tasks[t].op : -1);
    return STILES_ERR_PLAN;
  };
  auto in = [&](int64_t ref, int64_t lo_off, int64_t hi_off) {  // [ref+lo, ref+hi] inside its buffer
    if (ref < 0) return false;
    const int64_t off = ref & OFF_MASK;
    const int buf = (int)(ref >> BUF_SHIFT);
    return buf >= 0 && buf < 4 && ((allowed >> buf) & 1) && off + lo_off >= 0 && off + hi_off < lim;
  };
  for (int t = 0; t < nt; ++t) {
    const Task& tk = p.tasks[t];
    if (tk.op == OP_PREP) {  // a whole tile column of the base and of L, and the row-sum vectors
      const int64_t b = tk.ldo, a = tk.ldc, rows = (tk.flags & TF_CORNER) ? a : b;
      const int64_t len = (tk.flags & TF_CORNER) ? a * a : (1 + (int64_t)tk.zrows) * b * b + a * b;
      const int64_t base_lim = lim + 2 * (int64_t)tk.gcol;  // base values, then rb, ra
      auto in_base = [&](int64_t ref, int64_t lo_off, int64_t hi_off) {
        return ref >= 0 && (ref >> BUF_SHIFT) == BUF_A && (ref & OFF_MASK) + lo_off >= 0 &&
               (ref & OFF_MASK) + hi_off < base_lim;
      };
      if (tk.parts != 1 || !in(tk.out, 0, len - 1) || !in_base(tk.cin, 0, len - 1) ||
          !in_base(tk.aux, 0, rows - 1) || !in_base(tk.aux, tk.gcol, tk.gcol + rows - 1) ||
          (int64_t)tk.diag + rows > (int64_t)tk.gcol)
        return bad("PREP out of bounds", t);
      continue;
    }
    if (tk.op == OP_JOIN) {  // no work, no access
      if (tk.parts != 1 || tk.nseg != 0) return bad("join with work", t);
      continue;
    }
    if (tk.op == OP_ZERO) {  // zrows x n above the block
      if (tk.parts != 1 || tk.nseg != 0 || tk.zrows < 1 || tk.n < 1 ||
          !in(tk.out, -(int64_t)tk.zrows, -1 + (int64_t)(tk.n - 1) * tk.ldo))
        return bad("zeroed rows out of bounds", t);
      continue;
    }
    for (int q = 0; q < tk.parts; ++q) {
      int r0 = 0, c0 = 0, rm = tk.m, cn = tk.n;
      switch (tk.pmode) {
        case PM_ROWS2: r0 = 32 * q; rm = std::min(32, tk.m - r0); break;
        case PM_ROWS4: r0 = 16 * q; rm = std::min(16, tk.m - r0); break;
        case PM_QUAD4: r0 = 32 * (q & 1); c0 = 32 * (q >> 1); break;
        case PM_TRI3: r0 = q == 0 ? 0 : 32; c0 = q == 2 ? 32 : 0; break;
        case PM_TILE32: {
          const int pr = tk.m > 32 ? 2 : 1;
          r0 = 32 * (q % pr); c0 = 32 * (q / pr);
          break;
        }
        case PM_ROWS8: r0 = 8 * q; rm = std::min(8, tk.m - r0); break;
        case PM_TRI16: r0 = q == 0 ? 0 : 16; c0 = q == 2 ? 16 : 0; break;
        case PM_QUAD16: r0 = 16 * (q >> 1); c0 = 16 * (q & 1); break;
        default: break;
      }
      if (tk.pmode == PM_QUAD4 || tk.pmode == PM_TRI3 || tk.pmode == PM_TILE32) {
        rm = std::min(32, tk.m - r0); cn = std::min(32, tk.n - c0);
      } else if (tk.pmode == PM_TRI16 || tk.pmode == PM_QUAD16) {
        rm = std::min(16, tk.m - r0); cn = std::min(16, tk.n - c0);
      }
      if ((tk.pmode == PM_ROWS8 && tk.m > 32) || ((tk.pmode == PM_TRI16 || tk.pmode == PM_QUAD16) && (tk.m > 32 || tk.n > 32)))
        return bad("fine part mode on a block larger than 32", t);
      if ((tk.pmode == PM_TRI16 || tk.pmode == PM_QUAD16) && tk.prec != PREC_FP64)
        return bad("16 x 16 parts on a reduced-precision task", t);
      if (tk.prec == PREC_EMU64 && (rm > 32 || cn > 32)) return bad("emulated task part larger than 32 x 32", t);
      if (tk.prec != PREC_FP64 && tk.op != OP_UPD && tk.op != OP_NEG && tk.op != OP_STORE && tk.op != OP_SYMUPD)
        return bad("reduced precision on a triangular task", t);
      if (rm <= 0 || cn <= 0) continue;
      const int r1 = r0 + rm - 1, c1 = c0 + cn - 1;
      for (int g = tk.seg0; g < tk.seg0 + tk.nseg; ++g) {
        const Seg& sg = p.segs[g];
        if (sg.k <= 0) return bad("empty segment", t);
        const int64_t amax = (sg.trans & 1) ? (sg.k - 1) + (int64_t)r1 * sg.lda : r1 + (int64_t)(sg.k - 1) * sg.lda;
        const int64_t amin = (sg.trans & 1) ? (int64_t)r0 * sg.lda : r0;
        const int64_t bmax = (sg.trans & 2) ? c1 + (int64_t)(sg.k - 1) * sg.ldb : (sg.k - 1) + (int64_t)c1 * sg.ldb;
        const int64_t bmin = (sg.trans & 2) ? c0 : (int64_t)c0 * sg.ldb;
        if (!in(sg.a, amin, amax)) return bad("segment A out of bounds", t);
        if (!in(sg.b, bmin, bmax)) return bad("segment B out of bounds", t);
      }
      if (!in(tk.out, r0 + (int64_t)c0 * tk.ldo, r1 + (int64_t)c1 * tk.ldo)) return bad("output out of bounds", t);
      const bool uses_cin = tk.op == OP_UPD || tk.op == OP_POTRF || tk.op == OP_TRSM_RLT || tk.op == OP_SYMUPD;
      if (uses_cin && !in(tk.cin, r0 + (int64_t)c0 * tk.ldc, r1 + (int64_t)c1 * tk.ldc)) return bad("input out of bounds", t);
      if (tk.op == OP_TRSM_RLT && !in(tk.aux, 0, (tk.n - 1) + (int64_t)(tk.n - 1) * tk.ldx)) return bad("T out of bounds", t);
      if ((tk.op == OP_TRSM_LLN || tk.op == OP_TRTRI) && !in(tk.aux, 0, (tk.m - 1) + (int64_t)(tk.m - 1) * tk.ldx))
        return bad("T out of bounds", t);
      if (tk.op == OP_SYMUPD && !(tk.flags & TF_SYM_DIAG) &&
          !in(tk.aux, c0 + (int64_t)r0 * tk.ldx, c1 + (int64_t)r1 * tk.ldx))
        return bad("mirror out of bounds", t);
      if (tk.op == OP_POTRF && (tk.diag < 0 || tk.diag >= p.ndiag)) return bad("logdet slot out of range", t);
    }
  }
  // queue emulation: pushes per bucket / urgent queue never exceed capacity
  std::vector<int> rem(p.indeg), tail(p.tail0), seen(nt, 0);
  int utail = p.urgent_tail0;
  std::vector<int> stack;
  for (int t = 0; t < nt; ++t)
    if (p.indeg[t] == 0) stack.push_back(t);
  int done = 0;
  while (!stack.empty()) {
    const int t = stack.back();
    stack.pop_back();
    if (seen[t]++) return bad("task released twice", t);
    ++done;
    for (int e = p.succ_off[t]; e < p.succ_off[t + 1]; ++e) {
      const int sc = p.succ[e];
      if (sc < 0 || sc >= nt) return bad("successor out of range", t);
      if (--rem[sc] == 0) {
        const int parts = p.tasks[sc].parts;
        if (p.tasks[sc].flags & TF_URGENT) {
          utail += parts;
          if (utail > p.urgent_parts) return bad("urgent queue overflow", sc);
        } else {
          const int b = sc / kTasksPerBucket;
          tail[b] += parts;
          if (tail[b] > p.bcap[b] || tail[b] > kSlotsPerBucket) return bad("bucket overflow", sc);
        }
        stack.push_back(sc);
      }
      if (rem[sc] < 0) return bad("predecessor count underflow", sc);
    }
  }
  if (done != nt) return bad("some tasks never become ready", -1);
  for (int b = 0; b < p.nbuckets; ++b)
    if (tail[b] != p.bcap[b]) return bad("bucket not filled exactly", b * kTasksPerBucket);
  if (utail != p.urgent_parts) return bad("urgent queue not filled exactly", -1);
  return 0;
}


// ---------------------------------------------------------- race check ----
// Host check of a task table (tests): replays the table in its order (a
// topological order of the successor graph) and requires every two task
// parts that touch the same element, one of them writing it, to be ordered
// by the graph -- parts of one task run side by side, so they must not
// conflict at all. Accesses follow the kernel: each part reads its segments'
// operand regions, its input sub-block, the lower triangle of a triangular
// block, and writes its output sub-block (plus the mirror of SYMUPD and the
// rows above a ZERO task's block). Element granularity; plans of at most
// 16384 tasks. plant = 1 removes the predecessors of the last POTRF that has
// some (a planted race the check must find). serve: a request-server
// template, whose A is built in place in L (A references alias L) by PREP
// tasks that write their whole tile column of L (their reads of the shape's
// base values touch no buffer of the launch). Returns 0, STILES_ERR_PLAN (the
// first race printed to stderr) or STILES_ERR_INVALID_ARG.
namespace {

struct PartRect {
  int r0, c0, rm, cn;
};

PartRect part_rect(const Task& tk, int q) {
  PartRect x{0, 0, tk.m, tk.n};
  switch (tk.pmode) {
    case PM_ROWS2: x.r0 = 32 * q; x.rm = std::min(32, tk.m - x.r0); break;
    case PM_ROWS4: x.r0 = 16 * q; x.rm = std::min(16, tk.m - x.r0); break;
    case PM_ROWS8: x.r0 = 8 * q; x.rm = std::min(8, tk.m - x.r0); break;
    case PM_QUAD4: x.r0 = 32 * (q & 1); x.c0 = 32 * (q >> 1); break;
    case PM_TRI3: x.r0 = q == 0 ? 0 : 32; x.c0 = q == 2 ? 32 : 0; break;
    case PM_TRI16: x.r0 = q == 0 ? 0 : 16; x.c0 = q == 2 ? 16 : 0; break;
    case PM_QUAD16: x.r0 = 16 * (q >> 1); x.c0 = 16 * (q & 1); break;
    case PM_TILE32: {
      const int pr = tk.m > 32 ? 2 : 1;
      x.r0 = 32 * (q % pr);
      x.c0 = 32 * (q / pr);
      break;
    }
    default: break;
  }
  if (tk.pmode == PM_QUAD4 || tk.pmode == PM_TRI3 || tk.pmode == PM_TILE32) {
    x.rm = std::min(32, tk.m - x.r0);
    x.cn = std::min(32, tk.n - x.c0);
  } else if (tk.pmode == PM_TRI16 || tk.pmode == PM_QUAD16) {
    x.rm = std::min(16, tk.m - x.r0);
    x.cn = std::min(16, tk.n - x.c0);
  }
  return x;
}

class RaceCheck {
 public:
  RaceCheck(const Plan& p, int64_t lim, const std::vector<std::vector<int32_t>>& preds, bool serve)
      : p_(p), lim_(lim), n_((int)p.tasks.size()), words_((n_ + 63) / 64), serve_(serve) {
    anc_.assign((size_t)n_ * words_, 0ull);
    for (int t = 0; t < n_; ++t)
      for (int32_t q : preds[t]) {
        uint64_t* a = &anc_[(size_t)t * words_];
        const uint64_t* b = &anc_[(size_t)q * words_];
        for (int w = 0; w < words_; ++w) a[w] |= b[w];
        a[q >> 6] |= 1ull << (q & 63);
      }
    for (int b = 0; b < 4; ++b) {
      lw_[b].assign(lim, -1);
      head_[b].assign(lim, -1);
    }
  }
  bool before(int a, int b) const { return (anc_[(size_t)b * words_ + (a >> 6)] >> (a & 63)) & 1; }

  // one access of part `id` (4 task + part) to element `off` of buffer `buf`
  bool access(int buf, int64_t off, int id, bool write) {
    if (serve_ && buf == BUF_A) buf = BUF_L;  // a served request's A is built in place in L
    if (buf < 0 || buf > 3 || off < 0 || off >= lim_) return fail("access outside the buffers", id, -1, buf, off);
    const int t = id >> 2;
    const int w = lw_[buf][off];
    if (w >= 0 && w != id && !before(w >> 2, t)) return fail(write ? "unordered writes" : "read not ordered after the write", w, id, buf, off);
    if (!write) {
      // readers since the last write; one the new reader descends from is dropped
      // (a writer ordered after the new reader is ordered after it too)
      int* link = &head_[buf][off];
      while (*link >= 0) {
        const int r = pool_[*link].first;
        if (r == id) return true;
        if (r >> 2 != t && before(r >> 2, t)) *link = pool_[*link].second;
        else link = &pool_[*link].second;
      }
      pool_.push_back({id, head_[buf][off]});
      head_[buf][off] = (int)pool_.size() - 1;
      return true;
    }
    for (int e = head_[buf][off]; e >= 0; e = pool_[e].second) {
      const int r = pool_[e].first;
      if (r != id && !before(r >> 2, t)) return fail("write not ordered after a read", r, id, buf, off);
    }
    head_[buf][off] = -1;
    lw_[buf][off] = id;
    return true;
  }
  // rows r0 .. r0+rm-1 of columns c0 .. c0+cn-1 of the block at ref (leading dimension ld)
  bool rect(int64_t ref, int ld, int r0, int rm, int c0, int cn, int id, bool write, bool lower = false) {
    const int buf = (int)(ref >> BUF_SHIFT);
    const int64_t base = ref & OFF_MASK;
    for (int c = c0; c < c0 + cn; ++c)
      for (int r = r0; r < r0 + rm; ++r)
        if (!lower || r >= c)
          if (!access(buf, base + r + (int64_t)c * ld, id, write)) return false;
    return true;
  }
  bool task_part(int t, int q) {
    const Task& tk = p_.tasks[t];
    const int id = 4 * t + q;
    if (tk.op == OP_JOIN) return true;
    if (tk.op == OP_ZERO) return rect(tk.out, tk.ldo, -tk.zrows, tk.zrows, 0, tk.n, id, true);
    if (tk.op == OP_PREP) {  // the tile column of L (its base-value reads are outside the launch's buffers)
      const int64_t b = tk.ldo, a = tk.ldc;
      const int64_t len = (tk.flags & TF_CORNER) ? a * a : (1 + (int64_t)tk.zrows) * b * b + a * b;
      return len > 0 ? rect(tk.out, (int)len, 0, (int)len, 0, 1, id, true) : true;
    }
    const PartRect x = part_rect(tk, q);
    if (x.rm <= 0 || x.cn <= 0) return true;
    for (int g = tk.seg0; g < tk.seg0 + tk.nseg; ++g) {
      const Seg& sg = p_.segs[g];
      const bool ta = sg.trans & 1, tb = sg.trans & 2;
      // op(A) rows r0 .. r0+rm-1, op(B) columns c0 .. c0+cn-1, K = 0 .. k-1
      if (ta ? !rect(sg.a, sg.lda, 0, sg.k, x.r0, x.rm, id, false) : !rect(sg.a, sg.lda, x.r0, x.rm, 0, sg.k, id, false))
        return false;
      if (tb ? !rect(sg.b, sg.ldb, x.c0, x.cn, 0, sg.k, id, false) : !rect(sg.b, sg.ldb, 0, sg.k, x.c0, x.cn, id, false))
        return false;
    }
    const bool cin = tk.op == OP_UPD || tk.op == OP_POTRF || tk.op == OP_TRSM_RLT || tk.op == OP_SYMUPD;
    if (cin && !rect(tk.cin, tk.ldc, x.r0, x.rm, x.c0, x.cn, id, false)) return false;
    if (tk.op == OP_TRSM_RLT && !rect(tk.aux, tk.ldx, 0, tk.n, 0, tk.n, id, false, true)) return false;
    if ((tk.op == OP_TRSM_LLN || tk.op == OP_TRTRI) && !rect(tk.aux, tk.ldx, 0, tk.m, 0, tk.m, id, false, true))
      return false;
    if (!rect(tk.out, tk.ldo, x.r0, x.rm, x.c0, x.cn, id, true)) return false;
    if (tk.op == OP_SYMUPD && !((tk.flags & TF_SYM_DIAG) && x.r0 == x.c0)) {
      // the transpose of the sub-block: inside the same block, or the mirror block
      const bool dblk = tk.flags & TF_SYM_DIAG;
      if (!rect(dblk ? tk.out : tk.aux, dblk ? tk.ldo : tk.ldx, x.c0, x.cn, x.r0, x.rm, id, true)) return false;
    }
    return true;
  }
  bool fail(const char* what, int a, int b, int buf, int64_t off) {
    const int ta = a >= 0 ? a >> 2 : -1, tb = b >= 0 ? b >> 2 : -1;
    fprintf(stderr, "race_check: %s: task %d part %d (op %d) and task %d part %d (op %d), buffer %d element %lld\n",
            what, ta, a & 3, ta >= 0 ? (int)p_.tasks[ta].op : -1, tb, b & 3, tb >= 0 ? (int)p_.tasks[tb].op : -1,
            buf, (long long)off);
    return false;
  }

 private:
  const Plan& p_;
  int64_t lim_;
  int n_, words_;
  bool serve_;
  std::vector<uint64_t> anc_;
  std::vector<int> lw_[4], head_[4];
  std::vector<std::pair<int, int>> pool_;
};

}  // namespace

int race_check_plan(const Plan& p, int64_t lim, int plant, bool serve) {
  const int n = (int)p.tasks.size();
  if (n > 16384 || (int64_t)p.succ_off.size() != (int64_t)n + 1) return STILES_ERR_INVALID_ARG;
  std::vector<std::vector<int32_t>> preds(n);
  for (int t = 0; t < n; ++t)
    for (int e = p.succ_off[t]; e < p.succ_off[t + 1]; ++e) {
      const int s = p.succ[e];
      if (s <= t || s >= n) return STILES_ERR_PLAN;  // the table order must be topological
      preds[s].push_back(t);
    }
  if (plant == 1) {
    int victim = -1;
    for (int t = 0; t < n; ++t)
      if (p.tasks[t].op == OP_POTRF && !preds[t].empty()) victim = t;
    if (victim < 0) return STILES_ERR_INVALID_ARG;
    preds[victim].clear();
  }
  for (const Task& tk : p.tasks)
    if (tk.op == OP_PREP && !serve) return STILES_ERR_INVALID_ARG;
  RaceCheck rc(p, lim, preds, serve);
  for (int t = 0; t < n; ++t)
    for (int q = 0; q < std::max(1, (int)p.tasks[t].parts); ++q)
      if (!rc.task_part(t, q)) return STILES_ERR_PLAN;
  return 0;
}

}  // namespace stiles
