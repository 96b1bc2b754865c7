// Host-side check of the batched launch's item order (mcl::item_segments):
// every (session, local item) appears once, segments are contiguous and
// ordered, an interleaved session's segment is one of its (shortened) sweeps,
// a session alone on its map keeps its own sweeps in one segment, and the
// sessions on one map alternate round by round.
#include <cstdio>
#include <set>
#include <utility>
#include <vector>

#include "runtime.h"

using namespace mcl;

static int check(const std::vector<SegSession>& s, long long slots, bool inter, int max_rounds) {
  std::vector<int> sw;
  std::vector<ItemSeg> sg;
  const long long n = item_segments(s, slots, inter, max_rounds, &sw, &sg);
  long long total = 0;
  for (const SegSession& x : s) total += (long long)x.nblk * x.K;
  if (n != total) return printf("item count %lld, expected %lld\n", n, total), 1;
  if (sg.empty() || sg.back().begin != n || sg.back().session != -1) return printf("closing entry\n"), 1;
  std::set<std::pair<int, long long>> seen;
  for (size_t t = 0; t + 1 < sg.size(); ++t) {
    if (sg[t + 1].begin <= sg[t].begin) return printf("segments out of order\n"), 1;
    const int j = sg[t].session;
    const long long len = sg[t + 1].begin - sg[t].begin;
    int same = 0;
    for (const SegSession& x : s) same += x.values == s[j].values;
    if (!inter || same == 1) {
      if (sg[t].local0 != 0 || len != (long long)s[j].nblk * s[j].K || sw[j] != s[j].sweep)
        return printf("a session in order keeps its sweeps in one segment\n"), 1;
    } else {
      const long long per = (long long)sw[j] * s[j].K;
      if (sw[j] < 1 || sg[t].local0 % per != 0 || len > per) return printf("not one sweep\n"), 1;
    }
    for (long long i = 0; i < len; ++i)
      if (!seen.insert({j, sg[t].local0 + i}).second) return printf("item twice\n"), 1;
  }
  if ((long long)seen.size() != total) return printf("items missing\n"), 1;
  return 0;
}

int main() {
  int A = 1, B = 2, C = 3;
  const std::vector<std::vector<SegSession>> cases = {
      {{&A, 1954, 32, 19}, {&A, 1954, 32, 19}, {&A, 1954, 32, 19}, {&A, 1954, 32, 19}},
      {{&A, 7813, 32, 19}},
      {{&A, 8, 32, 8}, {&B, 500, 15, 40}, {&A, 1000, 32, 19}, {&C, 1, 1, 1}, {&B, 3, 15, 3}},
      {{&A, 100000, 2, 300}, {&A, 1, 32, 1}},
  };
  int bad = 0;
  for (const auto& c : cases)
    for (bool inter : {false, true})
      for (int max_rounds : {1, 64, 1024})
        for (long long slots : {1LL, 608LL, 100000LL}) bad |= check(c, slots, inter, max_rounds);
  // four equal sessions on one map, 608 slots: sweeps of 1954 / ceil(4 x 1954 x 32 / 608) blocks,
  // the sessions taking turns
  std::vector<int> sw;
  std::vector<ItemSeg> sg;
  item_segments(cases[0], 608, true, 1024, &sw, &sg);
  for (int k = 0; k < 8; ++k) bad |= sg[k].session != k % 4;
  bad |= sw[0] != 5;
  printf(bad ? "FAIL\n" : "ok\n");
  return bad;
}
