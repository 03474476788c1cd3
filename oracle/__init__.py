"""CPU oracle for the LEAD decoding path: test infrastructure, not product code.

Only the test-suite, the package smoke check and the benchmark's CPU-baseline leg may import
anything here. Every function is a plain, slow, readable restatement of the method in numpy,
written from the paper (LEAD, "A Local Ensemble-Assisted Parallel Decoding Framework for
Quantum Tanner Codes"), with FP64 for probabilities and LLRs. Where floating point decides an
integer (the hard decisions of the global min-sum decoder) the oracle takes that decision in
IEEE single precision with the operation order it documents, so that its decisions can be
compared bit for bit with a single-precision implementation.

Modules
  gf2      GF(2) linear algebra (RREF, rank, kernel, row-space membership)
  tanner   left-right Cayley complex, local views and the quantum Tanner code (Sec. II)
  philox   Philox4x32-10 counter RNG and the noise models (Sec. IV-A)
  local    exact local estimator of Phase 1 (coset weight enumerators, posteriors, ML decision)
  lead     Algorithm 1: local decoding + boost, regularised merge, global min-sum, failure check

Parity status: every function here is pinned by tests/test_oracle_*.py against closed forms,
brute force on small inputs, published test vectors or the paper's worked example, except the
global min-sum decoder beyond its textbook special cases (see lead.py).
"""
