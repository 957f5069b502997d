"""Plain, slow, CPU FP64 oracle for the Ski-LLS hot path (Cartis, Fiala & Shao,
"Hashing embeddings of optimal dimension, with applications to linear least
squares", arXiv 2105.11815).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The product path (the CUDA library and its Python binding) never imports,
links or calls anything here, and nothing here imports the product package.

Every function states the passage of the paper it follows.  Where the method
has a plain definition (the s-hashing matrix of Def. 5, the Walsh-Hadamard
matrix of Def. 8, the product S*A, the least-squares minimiser) the oracle
writes that definition out; where it is an iteration (LSQR in Step 4 of
Algorithm 1) the oracle takes the steps in the published order.

Modules
-------
hashing   counter-based draw of the s-hashing matrix (Def. 5) and of D (Def. 8)
sketch    S built entry by entry, S*A by rows, the s-hashing variant (Def. 7)
wht       Walsh-Hadamard butterflies and the HRHT premix H*D (Def. 8)
dht       the normalized Hartley transform and the HR-DHT premix F*D (Section 6)
qr        unblocked Householder QR of [SA | Sb] (Algorithm 1, Step 2), with column
          pivoting and the complete orthogonal form for rank-deficient sketches
lsqr      LSQR (Paige & Saunders) and the whole of Algorithm 1 (Ski-LLS), with
          plain QR or a rank-revealing Step 2
embedding subspace-embedding distortion (Lemma 2), coherence (Def. 6)
adjoint   gradient of x = argmin ||Ax-b|| with respect to A and b
"""
