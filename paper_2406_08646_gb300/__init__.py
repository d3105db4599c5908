"""GB300-native sparse SPD solver path: on-device COO assembly feeding a fused
Jacobi-preconditioned CG, with FP32-refined, batched and adjoint forms.

The compute path is the CUDA library ``libgbs.so`` (C-ABI declared in
``include/gbs.h``); :mod:`.binding` marshals arguments to it.  Importing this
package does not load the library; ``binding`` loads it on first use and raises
if it has not been built.
"""
__all__ = ["binding", "workloads"]
