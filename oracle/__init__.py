"""FP64 CPU oracle for the spin-free RIC-MRCCSD residual (test infrastructure).

Only tests/, `__graft_entry__.smoke()` and the CPU-baseline leg of bench.py may
import anything from this package.  It shares no code with the GPU library:
its equations come from its own spin-orbital generalized-Wick engine
(`oracle.wick`) and are evaluated unfactorised with numpy (`oracle.ricmrcc`).
`oracle.fockspace` is a brute-force Fock-space checker that pins the engine.
"""
