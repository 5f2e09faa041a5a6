"""CPU oracle of the query-pipeline hot path and of the cost-model network.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.
"""
