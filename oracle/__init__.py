"""Plain FP64 CPU oracle of the perfect-dispersion 3D EM-PIC step.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the CPU
baseline leg of bench.py.  The product path (the CUDA library and its Python
binding) never imports it.
"""
