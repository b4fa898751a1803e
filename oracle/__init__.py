"""FP64 CPU oracle for the QR-based C3v CTMRG step (TEST INFRASTRUCTURE).

Only tests, the smoke check and the benchmark's CPU-baseline leg may import it.
"""
