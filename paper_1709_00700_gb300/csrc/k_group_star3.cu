// Grouped join shape of the SSB Q3 flight (Section 9.2.1): three probes into
// filtered build-side tables, grouping on the three payloads they bind, one
// SUM over a fact column.
#include "k_group.cuh"

namespace pv {

using ShStar3 = Shape<Cols<TI32, TI32, TI32, TI64>, Where<>, Probes<0, 1, 2>, Key<PL<0, 0>, PL<1, 0>, PL<2, 0>>,
                      Aggs<Sum<Mul<X<3>>>>, Proj<>>;

void register_group_star3() { reg_grouped<ShStar3, 1>(); }

}  // namespace pv
