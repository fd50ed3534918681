"""FP64 CPU oracle of the msDEM model.  Test infrastructure only: imported by
tests/, the smoke check and the CPU-baseline leg of bench.py, never by the
product package."""
