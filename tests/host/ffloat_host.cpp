// Host driver of the float-float helpers of the reaction kernels: reads
// doubles from stdin, one per line, and prints for each the split (ok flag,
// hi, lo as hex floats), the widened hi, and the sum, the product
// and the product with hi of the pair with itself in float-float arithmetic,
// and the float nearest to the double.
#include <cstdio>

#include "ffloat.cuh"

using namespace kfbi::ffl;

int main() {
  double x;
  while (std::scanf("%lf", &x) == 1) {
    ff p{0.0f, 0.0f};
    const bool ok = split(x, p);
    const ff s = add(p, p), q = mul(p, p), r = mul(p, p.h);
    std::printf("%d %a %a %a %a %a %a %a %a %a %a\n", ok ? 1 : 0, (double)p.h, (double)p.l, widen(p.h), (double)s.h,
                (double)s.l, (double)q.h, (double)q.l, (double)r.h, (double)r.l, (double)narrow(x));
  }
  return 0;
}
