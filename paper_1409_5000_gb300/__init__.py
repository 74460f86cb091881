"""GB300-native summed total communicability (arXiv 1409.5000).

Scores every node of one or more graphs by the Estrada-Benzi total
communicability e^A 1 (paper eq. 4), computed with an m-step Lanczos
(Krylov) approximation, sums the scores over N background realisations
that share one embedded target (eq. 5), and returns the top-k nodes.

All compute runs in the CUDA library ``_lib/libcb.so`` (sm_103a); the
Python layer in :mod:`.binding` only marshals arguments.  Importing the
package does not load the library; the first call does, and it raises if
the library is missing.
"""

__all__ = ["binding", "synth"]
