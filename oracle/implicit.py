"""The implicit operator of one zip-up einsumsvd step (oracle side).

Algorithm 3's einsumsvd line refactorises the network (carry V, old boundary
site S, MPO site O) into two sites joined by one truncated bond.  In the
two-layer form (Sec. III-B) the MPO site is a ket site K and a bra site Kb
sharing the physical index s, so the matrix being factorised is

  A[(k,t), (x,X,b,e,E)] = sum_{a,l,L,u,U,s}
        V[k,t,a,(l,L)] * S[a,(u,U),b] * K[s,l,u,x,e] * conj(Kb[s,L,U,X,E])

with rows (k, t) = (left bond of the carry, down pair of the previous
column) and columns (x, X, b, e, E) = (ket/bra down bond, old boundary right
bond, ket/bra right bond).  Following Sec. IV-A, A is never formed: A X and
A^H Y are contractions of the uncontracted network with the block X or Y.
The one-layer case is the same operator with a trivial bra (all dims 1,
value 1) and d = 1.

Layouts: V [kL][t][a][h] with h = l*DL + L; S [a][v][b] with v = u*DU + U;
K and Kb [d][left][up][down][right].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch


def _common(*arrays):
    """The operands as CPU torch tensors of one FP64 type (complex128 if any
    operand is complex), sharing memory with the NumPy arrays where possible."""
    cplx = any(np.iscomplexobj(a) for a in arrays)
    dt = np.complex128 if cplx else np.float64
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=dt)) for a in arrays]


@dataclass
class ImplicitOp:
    V: np.ndarray      # [kL][t][a][h]
    S: np.ndarray      # [a][v][b]
    K: np.ndarray      # [d][l][u][x][e]
    Kb: np.ndarray     # [d][L][U][X][E]

    def __post_init__(self):
        d, Dl, Du, Dx, De = self.K.shape
        db, DL, DU, DX, DE = self.Kb.shape
        assert d == db
        kL, t, a, h = self.V.shape
        a2, v, b = self.S.shape
        assert a == a2 and h == Dl * DL and v == Du * DU
        self.dims = dict(d=d, Dl=Dl, Du=Du, Dx=Dx, De=De, DL=DL, DU=DU,
                         DX=DX, DE=DE, kL=kL, t=t, a=a, b=b)
        self.V6 = self.V.reshape(kL, t, a, Dl, DL)
        self.S4 = self.S.reshape(a, Du, DU, b)
        self.M = kL * t
        self.N = Dx * DX * b * De * DE
        self.col_shape = (Dx, DX, b, De, DE)

    @property
    def is_complex(self):
        return any(np.iscomplexobj(x) for x in (self.V, self.S, self.K, self.Kb))

    def matvec(self, X: np.ndarray) -> np.ndarray:
        """A X for X of shape (N, ell) -> (M, ell).

        Pairwise contractions in the cheap order of Table 2's two-layer
        column: ket, bra (the two d D^6 terms), then S and V (the m^2 terms).
        Each pairwise sum is one torch.einsum on the CPU (FP64 arithmetic).
        """
        ell = X.shape[1]
        X, K, Kb, S4, V6 = _common(X, self.K, self.Kb, self.S4, self.V6)
        X6 = X.reshape(*self.col_shape, ell)
        T1 = torch.einsum("xXbeEj,sluxe->XbEjslu", X6, K)
        T2 = torch.einsum("XbEjslu,sLUXE->bjluLU", T1, Kb.conj())
        del T1
        T3 = torch.einsum("bjluLU,auUb->jlLa", T2, S4)
        del T2
        Y = torch.einsum("jlLa,ktalL->ktj", T3, V6)
        return Y.reshape(self.M, ell).resolve_conj().numpy()

    def rmatvec(self, Y: np.ndarray) -> np.ndarray:
        """A^H Y for Y of shape (M, ell) -> (N, ell), the chain reversed."""
        ell = Y.shape[1]
        Y, K, Kb, S4, V6 = _common(Y, self.K, self.Kb, self.S4, self.V6)
        Y3 = Y.reshape(self.dims["kL"], self.dims["t"], ell)
        Z3 = torch.einsum("ktj,ktalL->jalL", Y3, V6.conj())
        Z2 = torch.einsum("jalL,auUb->jlLuUb", Z3, S4.conj())
        Z1 = torch.einsum("jlLuUb,sluxe->jLUbsxe", Z2, K.conj())
        del Z2
        X = torch.einsum("jLUbsxe,sLUXE->xXbeEj", Z1, Kb)
        return X.reshape(self.N, ell).resolve_conj().numpy()

    def dense(self) -> np.ndarray:
        """The explicit M x N matrix (only for checks on small shapes)."""
        A = np.einsum("ktalL,auUb,sluxe,sLUXE->ktxXbeE",
                      self.V6, self.S4, self.K, np.conj(self.Kb),
                      optimize="greedy")
        return A.reshape(self.M, self.N)

    def product_macs(self, ell: int) -> int:
        """Multiply-adds of one product in the contraction order of Table 2's
        two-layer IBMPS column: two D^6 stages, then the two m^2 stages."""
        g = self.dims
        s1 = ell * g["b"] * g["d"] * g["Dl"] * g["Du"] * g["Dx"] * g["De"] * g["DX"] * g["DE"]
        s2 = ell * g["b"] * g["d"] * g["Dl"] * g["Du"] * g["DL"] * g["DU"] * g["DX"] * g["DE"]
        s3 = ell * g["a"] * g["b"] * g["Dl"] * g["DL"] * g["Du"] * g["DU"]
        s4 = ell * g["kL"] * g["t"] * g["a"] * g["Dl"] * g["DL"]
        return s1 + s2 + s3 + s4
