// Grouped shape: low-cardinality fixed-point aggregation (date filter, two
// one-byte group codes, 8 aggregates of products), the compute-heavy
// aggregation pipeline of Section 9.2.1.
#include "k_group.cuh"

namespace pv {

using ShLowcard =
    Shape<Cols<TI32, TU8, TU8, TI64, TI64, TI64, TI64>, Where<P<0>>, Probes<>, Key<X<1>, X<2>>,
          Aggs<Sum<Mul<X<3>>>, Sum<Mul<X<4>>>, Sum<Mul<X<5>>>, Sum<Mul<X<6>>>, Sum<Mul<X<4>, CMX<5, 0>>>,
               Sum<Mul<X<4>, CMX<5, 1>, XPC<6, 2>>>, Sum<Mul<X<3>, X<4>>>, Count>,
          Proj<>>;

void register_group_lowcard() { reg_grouped<ShLowcard, 1>(); }

}  // namespace pv
