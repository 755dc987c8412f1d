"""FP64 CPU oracle for the splattable-neural-primitive rasterizer (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It never imports the CUDA package and the CUDA package never
imports it; the two share only the seeded inputs of paper_2510_08491_gb300.synth.

Every function here that is not pinned to an independent check says
"parity unpinned" in its docstring.
"""
