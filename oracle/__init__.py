"""FP64 CPU oracle for the state-vector hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
leg may import this package.  It shares no code with the CUDA library
(paper_2010_09746_gb300); the two meet only through the seeded circuit
generators in workloads/, which contain no simulation arithmetic.

Parity pins live in tests/test_oracle_*.py (not GPU).  Every routine here is
pinned by at least one check that does not re-use the routine itself: dense
2^n x 2^n matrix products built entry by entry, closed forms (GHZ, QFT of a
basis state), brute-force storage indices, and the paper's printed statistics.
"""
