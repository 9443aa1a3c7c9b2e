// Host-side race check of the factorisation's two-stream schedule.
//
// The factor ops run on two streams whose only cross-stream ordering is the
// event each op may wait for.  This check enumerates, element by element of
// the arena, what every op reads and writes (exactly the entries that can
// change a result: GEMM operand rows / columns of unmasked outputs, copied
// and masked entries, panel blocks, extend-add maps) and replays the ops in
// list order with a vector clock per op.  Two accesses to one element from
// different streams, at least one a write, must be ordered by the clocks;
// every unordered pair is a race.  Runs on symbolic plans (no device).
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "plan.hpp"

namespace cl {

namespace {

struct Tracker {
  const std::vector<Op>& ops;
  std::vector<int> lw;                   // last writer op, -1 none
  std::vector<int> lr0, lr1;             // per stream: largest sequence number of a read since the last write
  std::vector<int> seq;                  // op -> sequence number on its stream (1-based)
  std::vector<std::array<int, 2>> vc;    // op -> vector clock
  long long conflicts = 0;
  std::string first;
  int cur = -1;
  Tracker(const std::vector<Op>& o, int64_t n) : ops(o), lw(n, -1), lr0(n, 0), lr1(n, 0) {}

  bool hb(int a, int b) const { return vc[b][ops[a].stream] >= seq[a]; }
  void report(const char* what, int64_t e, int other) {
    if (conflicts++ == 0) {
      char buf[256];
      std::snprintf(buf, sizeof(buf), "%s at element %lld: op %d (kind %d, stream %d) vs op %d (kind %d, stream %d)",
                    what, (long long)e, cur, (int)ops[cur].kind, ops[cur].stream, other,
                    other >= 0 ? (int)ops[other].kind : -1, other >= 0 ? ops[other].stream : -1);
      first = buf;
    }
  }
  // phase 0: check against earlier ops; phase 1: record
  int phase = 0;
  void read(int64_t e) {
    const int s = ops[cur].stream;
    if (phase == 0) {
      if (lw[e] >= 0 && lw[e] != cur && !hb(lw[e], cur)) report("read after unordered write", e, lw[e]);
    } else {
      int& r = s ? lr1[e] : lr0[e];
      if (seq[cur] > r) r = seq[cur];
    }
  }
  void write(int64_t e) {
    const int s = ops[cur].stream;
    if (phase == 0) {
      if (lw[e] >= 0 && lw[e] != cur && !hb(lw[e], cur)) report("write after unordered write", e, lw[e]);
      const int other = 1 - s;
      const int r = other ? lr1[e] : lr0[e];
      if (r > vc[cur][other]) report("write after unordered read", e, -1);
    } else {
      lw[e] = cur;
      lr0[e] = lr1[e] = 0;
    }
  }
};

template <typename R, typename W>
void copy_footprint(const Plan& p, int d0, int d1, R& visit_read, W& visit_write) {
  for (int d = d0; d < d1; ++d) {
    const CopyDesc& x = p.copies[d];
    for (int i = 0; i < x.rows; ++i)
      for (int j = 0; j < x.cols; ++j) {
        if (x.rmask.hit(i) || x.cmask.hit(j)) continue;
        visit_read(x.src + (int64_t)i * x.lds + j);
        visit_write(x.dst + (int64_t)i * x.ldd + j);
      }
  }
}

template <typename R, typename W>
void footprint(const Plan& p, const Op& op, R&& visit_read, W&& visit_write) {
  switch (op.kind) {
    case OP_ZERO:
    case OP_ASSEMBLE:
      for (int64_t e = 0; e < p.pool_elems; ++e) visit_write(e);
      break;
    case OP_EXTADD:
      for (int d = op.d0; d < op.d1; ++d) {
        const ExtAddDesc& x = p.extadd[d];
        for (int i = 0; i < x.nfp; ++i)
          for (int j = 0; j < x.nfp; ++j) {
            bool any = false;
            for (int q = 0; q < x.nchild; ++q) {
              const int ci = p.maps[x.map[q] + i / 3], cj = p.maps[x.map[q] + j / 3];
              if (ci < 0 || cj < 0) continue;
              visit_read(x.child[q] + (int64_t)(x.kc[q] + 3 * ci + i % 3) * x.nfc[q] + x.kc[q] + 3 * cj + j % 3);
              any = true;
            }
            if (any) {
              visit_read(x.parent + (int64_t)i * x.nfp + j);
              visit_write(x.parent + (int64_t)i * x.nfp + j);
            }
          }
      }
      break;
    case OP_PANEL:  // the candidate rows in the panel's columns (inverse of the chosen block, displaced rows)
      for (int d = op.d0; d < op.d1; ++d) {
        const PanelDesc& x = p.panels[d];
        for (int i = 0; i < x.nc; ++i)
          for (int j = 0; j < x.bp; ++j) {
            visit_read(x.a + (int64_t)i * x.ld + j);
            visit_write(x.a + (int64_t)i * x.ld + j);
          }
      }
      copy_footprint(p, op.x0, op.x1, visit_read, visit_write);  // the copies launched with the panels
      break;
    case OP_SWAP:  // the candidate rows in every column outside the panel
      for (int d = op.d0; d < op.d1; ++d) {
        const PanelDesc& x = p.panels[d];
        if (x.nc <= x.bp) continue;
        const int64_t row0 = x.a - x.col0;  // column 0 of the panel's first row
        for (int i = 0; i < x.nc; ++i)
          for (int j = 0; j < x.ld; ++j) {
            if (j >= x.col0 && j < x.col0 + x.bp) continue;
            visit_read(row0 + (int64_t)i * x.ld + j);
            visit_write(row0 + (int64_t)i * x.ld + j);
          }
      }
      break;
    case OP_GEMM:
      for (int d = op.d0; d < op.d1; ++d) {
        const GemmDesc& g = p.gemm[d];
        std::vector<int> rows, cols;
        for (int r = 0; r < g.M; ++r)
          if (!g.rmask.hit(r)) rows.push_back(r);
        for (int c = 0; c < g.N; ++c)
          if (!g.cmask.hit(c)) cols.push_back(c);
        if (rows.empty() || cols.empty()) continue;
        auto ai = [&g](int r, int k) { return g.a + ((g.trans & 1) ? (int64_t)k * g.lda + r : (int64_t)r * g.lda + k); };
        auto bi = [&g](int k, int c) { return g.b + ((g.trans & 2) ? (int64_t)c * g.ldb + k : (int64_t)k * g.ldb + c); };
        auto ci = [&g](int r, int c) { return g.c + ((g.trans & 4) ? (int64_t)c * g.ldc + r : (int64_t)r * g.ldc + c); };
        for (int r : rows)
          for (int k = 0; k < g.K; ++k) visit_read(ai(r, k));
        for (int k = 0; k < g.K; ++k)
          for (int c : cols) visit_read(bi(k, c));
        for (int r : rows)
          for (int c : cols) {
            if (g.beta) visit_read(ci(r, c));
            visit_write(ci(r, c));
          }
      }
      break;
    case OP_COPY:
      copy_footprint(p, op.d0, op.d1, visit_read, visit_write);
      break;
    default:
      break;
  }
}

}  // namespace

long long check_factor_schedule(const Plan& p, bool ignore_waits, std::string* first) {
  const auto& ops = p.factor_ops;
  Tracker t(ops, p.arena_elems);
  t.seq.resize(ops.size());
  t.vc.resize(ops.size());
  int nseq[2] = {0, 0};
  std::array<int, 2> last[2] = {{0, 0}, {0, 0}};
  for (size_t i = 0; i < ops.size(); ++i) {
    const int s = ops[i].stream;
    t.seq[i] = ++nseq[s];
    std::array<int, 2> v = last[s];
    v[s] = t.seq[i];
    if (!ignore_waits && ops[i].wait >= 0) {
      const auto& w = t.vc[ops[i].wait];
      v[0] = std::max(v[0], w[0]);
      v[1] = std::max(v[1], w[1]);
    }
    t.vc[i] = v;
    last[s] = v;
  }
  for (size_t i = 0; i < ops.size(); ++i) {
    t.cur = (int)i;
    // phase 0 checks every access against earlier ops, phase 1 records them
    // (an op that reads and writes one element does not conflict with itself)
    for (t.phase = 0; t.phase < 2; ++t.phase)
      footprint(p, ops[i], [&](int64_t e) { t.read(e); }, [&](int64_t e) { t.write(e); });
  }
  if (first) *first = t.first;
  return t.conflicts;
}

}  // namespace cl
