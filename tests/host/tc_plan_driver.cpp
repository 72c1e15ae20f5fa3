// Host-side driver for the grouped tensor-core launch planning helpers of
// tcgemm.h (work-item expansion, segment weights, alpha merge classes).
// Reads commands from stdin, prints results; used by test_host_tc_plan.py.
#include <cstdio>
#include <string>
#include <vector>

#include "tcgemm.h"

int main() {
  char mode[32];
  while (std::scanf("%31s", mode) == 1) {
    const std::string m(mode);
    if (m == "items") {
      int nc = 0, no = 0, ns = 0;
      std::vector<TcCluster> cl;
      std::vector<TcGroupOp> ops;
      std::vector<TcSeg> segs;
      if (std::scanf("%d", &nc) != 1) return 1;
      for (int i = 0; i < nc; ++i) {
        TcCluster c{};
        long long b;
        if (std::scanf("%lld %d %d %d %d %d %d %d", &b, &c.op0, &c.nops, &c.mt, &c.kt_total, &c.kps, &c.ksplit,
                       &c.W) != 8)
          return 1;
        c.begin = b;
        cl.push_back(c);
      }
      if (std::scanf("%d", &no) != 1) return 1;
      for (int i = 0; i < no; ++i) {
        TcGroupOp o{};
        if (std::scanf("%d %d %d %d", &o.nt, &o.nseg, &o.seg0, &o.kt0) != 4) return 1;
        ops.push_back(o);
      }
      if (std::scanf("%d", &ns) != 1) return 1;
      for (int i = 0; i < ns; ++i) {
        TcSeg s{};
        if (std::scanf("%d", &s.kt) != 1) return 1;
        segs.push_back(s);
      }
      std::vector<TcItem> items;
      if (!tc_expand_items(cl, ops, segs, items)) {
        std::printf("overflow\n");
        continue;
      }
      std::printf("ok %zu\n", items.size());
      for (const TcItem& it : items)
        std::printf("%d %d %d %d %d %d %d %d\n", it.oi, it.mi, it.ni, it.kt0, it.kt1, it.s0, it.s1, it.send);
    } else if (m == "weights") {
      int n = 0;
      if (std::scanf("%d", &n) != 1 || n < 1 || n > 64) return 1;
      std::vector<double> a(n);
      for (double& x : a)
        if (std::scanf("%lf", &x) != 1) return 1;
      uint8_t code[kTcMaxSeg] = {};
      float base = 0.f;
      if (!tc_segment_weights(a.data(), n, code, &base)) {
        std::printf("bad\n");
        continue;
      }
      std::printf("ok %.9g", base);
      for (int i = 0; i < n; ++i) std::printf(" %d", code[i]);
      std::printf("\n");
    } else if (m == "class") {
      double a = 0;
      if (std::scanf("%lf", &a) != 1) return 1;
      std::string key;
      tc_alpha_class(a, key);
      std::printf("key ");
      for (unsigned char ch : key) std::printf("%02x", ch);
      std::printf("\n");
    } else {
      return 1;
    }
  }
  return 0;
}
