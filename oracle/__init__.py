"""FP64 CPU oracle for the reacting Navier-Stokes hot path (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py may import this
package. It shares no code with the CUDA library and imports nothing from it; the only module both
sides use is the seeded input generator ``paper_2210_05547_gb300.inputs``.
"""
