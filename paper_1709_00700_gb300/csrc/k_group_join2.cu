// Grouped join shapes of the Table 2 pipeline programs: filter, two probes,
// grouping on the payload of the first or of the second build.
#include "k_group.cuh"

namespace pv {

using ShTable2X = Shape<Cols<TI32, TI32, TI32, TI64>, Where<P<0>>, Probes<1, 2>, Key<PL<0, 0>>,
                        Aggs<Sum<Mul<X<3>>>, Count>, Proj<>>;
using ShTable2Y = Shape<Cols<TI32, TI32, TI32, TI64>, Where<P<0>>, Probes<1, 2>, Key<PL<1, 0>>,
                        Aggs<Sum<Mul<X<3>>>, Count, Min<Mul<X<3>>>, Max<Mul<X<3>>>>, Proj<>>;

void register_group_join2() {
  reg_grouped<ShTable2X, 1>();
  reg_grouped<ShTable2Y, 1>();
}

}  // namespace pv
