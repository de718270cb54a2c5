"""FP64 CPU oracle for the TTN-HEOM hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, readable restatement of the method of the TENSO
paper (arXiv 2603.17711) in numpy float64/complex128. It exists to check the
CUDA path: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import it. The product path never imports, links or calls
anything in here, and nothing in here imports the product package.

Modules
  bcf    -- bath-correlation features (Sec. 2.1, Eqs. 2-3, Eq. bcfdecores,
            Eq. DL, Eq. BO; Pade decomposition of the Bose function).
  sop    -- the 5K+2 sum-of-products terms of the bexcitonic HEOM generator
            (Eq. heom-std, Eq. dissipator, Eq. master_lvn) with a metric choice
            (Sec. 7.4, Listing custommetric).
  dense  -- brute-force dense hierarchy: dOmega/dt = L Omega on the full
            M*M*prod(N_k) vector (Eq. EDO-eom).
  ttn    -- tree tensor network state, environments, effective operators,
            Householder QR, RK4, the fixed-rank (ps1) and adaptive-rank (ps2)
            projector-splitting steps and the reduced density matrix
            (Sec. 2.3, Eq. omega_tensor, Eq. semiunitary, Sec. 2.3 last paragraph).

Parity status of each function is stated in its docstring: "pinned by ..."
names the independent check in tests/ that fixes it.
"""
