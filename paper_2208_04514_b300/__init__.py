"""DAWN (Feng et al., ICS '24) hot path on B300: exact unweighted shortest paths
as a level-synchronous Boolean vector-matrix product over (OR, AND).

``paper_2208_04514_b300.dawn`` is the thin Python binding of the C ABI in
``include/dawn.h``; ``paper_2208_04514_b300.graphgen`` draws the seeded
synthetic graphs.
"""
