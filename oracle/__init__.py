"""Plain, slow FP64 CPU oracle of the gPEPS simple-update Trotter evolution.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` use it.  It shares no code with the CUDA path;
both read their inputs from ``workloads``.

Modules
-------
graph        edge colouring (update order) and leg order of every site
su           simple update + mean-field <Z> (paper, section "Method"; Eqs. 2-3)
statevector  brute-force state vectors of the kicked Ising circuit (Eqs. 2-3)
pauli        Clifford Pauli propagation at theta_h = pi/2 (App. B, Eqs. 4-7)
lightcone    exact <Z_q> from the backward light cone of q (App. C argument)
weight       Weight-N observables by Clifford back-evolution (App. B)
bp           belief-propagation regauging after a Trotter step ("Method", "Benchmarking")

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against values that do not come from the oracle itself (see each module).
"""
