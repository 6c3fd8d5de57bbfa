"""CPU oracle for the encrypted CSSC SpMV (TEST INFRASTRUCTURE ONLY).

A plain, slow, obviously correct CPU implementation of what the GPU path
computes: the BGV-RNS scheme the SpMV runs under, the CSSC format
(Algorithm 5), chunk generation (Algorithm 2), vector reorganisation
(Algorithm 3), the cloud evaluation of Algorithm 1 and the aggregation of
Algorithm 4.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it and shares no code with it: the prime
search, root selection, RNS constants, transforms, samplers, format
conversion and the key switch are all written separately here.

Exact arithmetic: every modular product is a 128-bit product reduced with
``%`` (``he_oracle.c``) or a Python integer; CRT reconstruction uses Python
big integers.

Pinned (see ``tests/test_oracle_*.py``): NTT vs its O(N^2) definition and vs
schoolbook negacyclic convolution; batch encoding vs direct evaluation at the
roots; base conversion vs big-integer CRT; key switching / rotation /
relinearisation vs decryption invariants and noise bounds; CSSC vs a dense
round trip and the Figure 5 example; numBits vs Section 4.5; totalSum vs a
brute-force slot simulation; op counts vs Table 3; end to end vs plaintext
A.x.  Parity unpinned: the byte counts of the client-to-client message
(Table 5, A->B column) and the Figure 4/6/7 example beyond its rList.
"""
