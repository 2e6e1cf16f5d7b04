"""The oracle: a plain, slow, FP64 CPU restatement of the paper's method.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import anything from this package.  It shares no
code with the CUDA library and never imports it.
"""
