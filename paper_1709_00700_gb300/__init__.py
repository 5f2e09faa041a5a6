"""GB300-native query-pipeline variants (scan, filter, hash probe, grouped
aggregation, projection compaction) behind the ``libpv`` C-ABI library.

The CUDA library is loaded on first use by :mod:`paper_1709_00700_gb300.pv`;
importing the package itself loads no native code.
"""
__all__ = ["datagen", "workloads", "pv"]
