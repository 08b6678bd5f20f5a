"""FP64 CPU oracle of the coherent hyperspin machine (arXiv 2308.02329).

TEST INFRASTRUCTURE ONLY: the independent oracle for the CUDA path.  Only the
test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import it.  It shares no code with ``paper_2308_02329_gb300``.
"""
