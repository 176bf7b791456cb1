"""FP64 CPU oracle for the PIC/FDTD-Drude time step, and the thin-film theory.

Test infrastructure only: tests, ``__graft_entry__.smoke()`` and the bench's
CPU-baseline leg may import this package.  The CUDA product path never does.
"""
