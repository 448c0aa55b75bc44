"""Learned prefilter: the binding of pastis_pair_features / pastis_mlp_* /
pastis_prefilter_select and the training driver around them.

Every numeric step (features, forward, backward, Adam, selection) runs in the library's
kernels; this module allocates the caller-owned parameter buffers with torch, sequences
the calls and picks the decision threshold.  Labels come from the exact path (the
`passes` verdict of pastis_align_pairs), against which edge recall is also measured.
"""
import ctypes
import math

import numpy as np
import torch

from . import pastis as _p

FEAT, HID = 16, 256
NW1, NW2, NW3 = FEAT * HID, HID * HID, HID
NPARAM = NW1 + HID + NW2 + HID + NW3 + 1


class c_mlp(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("w2", ctypes.c_void_p), ("b2", ctypes.c_void_p),
                ("w3", ctypes.c_void_p), ("b3", ctypes.c_void_p), ("w1b", ctypes.c_void_p), ("w2b", ctypes.c_void_p),
                ("w3b", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("adam_m", ctypes.c_void_p),
                ("adam_v", ctypes.c_void_p), ("step", ctypes.c_int64)]


def _lib():
    L = _p.lib()
    if not getattr(L, "_mlp_sigs", False):
        P, i64 = ctypes.c_void_p, ctypes.c_int64
        L.pastis_pair_features.argtypes = [P, P, P, P, i64, ctypes.POINTER(_p.c_params), P]
        L.pastis_pair_features.restype = ctypes.c_int32
        L.pastis_pair_features_qt.argtypes = [P, P, P, P, P, P, i64, ctypes.POINTER(_p.c_params), P]
        L.pastis_pair_features_qt.restype = ctypes.c_int32
        L.pastis_mlp_forward.argtypes = [P, ctypes.POINTER(c_mlp), P, i64, P]
        L.pastis_mlp_forward.restype = ctypes.c_int32
        L.pastis_mlp_train_step.argtypes = [P, ctypes.POINTER(c_mlp), P, P, i64, ctypes.c_float, ctypes.c_float, P]
        L.pastis_mlp_train_step.restype = ctypes.c_int32
        L.pastis_prefilter_select.argtypes = [P, P, P, i64, ctypes.c_float, P, i64, ctypes.POINTER(i64)]
        L.pastis_prefilter_select.restype = ctypes.c_int32
        L._mlp_sigs = True
    return L


class MLP:
    """Parameters of the 16-256-256-1 network in caller-owned device buffers."""

    def __init__(self, device="cuda", seed=0):
        g = torch.Generator().manual_seed(seed)
        self.device = torch.device(device)

        def init(shape, fan_in):
            return (torch.randn(shape, generator=g) * math.sqrt(2.0 / fan_in)).float().to(self.device)

        self.w1 = init((FEAT, HID), FEAT)
        self.b1 = torch.zeros(HID, device=self.device)
        self.w2 = init((HID, HID), HID)
        self.b2 = torch.zeros(HID, device=self.device)
        self.w3 = init((HID,), HID) * 0.1
        self.b3 = torch.zeros(1, device=self.device)
        self.w1b = self.w1.to(torch.bfloat16)
        self.w2b = self.w2.to(torch.bfloat16)
        self.w3b = self.w3.to(torch.bfloat16)
        self.grad = torch.zeros(NPARAM, device=self.device)
        self.adam_m = torch.zeros(NPARAM, device=self.device)
        self.adam_v = torch.zeros(NPARAM, device=self.device)
        self.step = 0

    def c(self) -> c_mlp:
        m = c_mlp()
        for f in ("w1", "b1", "w2", "b2", "w3", "b3", "w1b", "w2b", "w3b", "grad", "adam_m", "adam_v"):
            setattr(m, f, getattr(self, f).data_ptr())
        m.step = self.step
        return m

    def state_dict(self):
        return {k: getattr(self, k).detach().cpu().clone() for k in
                ("w1", "b1", "w2", "b2", "w3", "b3", "w1b", "w2b", "w3b", "adam_m", "adam_v")} | {"step": self.step}

    def load_state_dict(self, sd):
        for k, v in sd.items():
            if k == "step":
                self.step = int(v)
            else:
                getattr(self, k).copy_(v.to(self.device))

    def grads(self):
        """Views of the gradient buffer: w1, b1, w2, b2, w3, b3."""
        g, o = self.grad, 0
        out = []
        for n, shape in ((NW1, (FEAT, HID)), (HID, (HID,)), (NW2, (HID, HID)), (HID, (HID,)), (NW3, (HID,)), (1, (1,))):
            out.append(g[o:o + n].view(shape))
            o += n
        return out


def features(ctx, codes, offsets, pairs, params) -> torch.Tensor:
    n = pairs.shape[0]
    x = torch.empty((max(n, 1), FEAT), dtype=torch.bfloat16, device=codes.device)
    p = params.c()
    _p._check("pastis_pair_features", _lib().pastis_pair_features(
        ctx.h, _p._ptr(codes), _p._ptr(offsets), _p._ptr(pairs), n, ctypes.byref(p), _p._ptr(x)))
    return x[:n]


def features_qt(ctx, qcodes, qoffsets, tcodes, toffsets, pairs, params) -> torch.Tensor:
    """Features of query x target candidates (serving form)."""
    n = pairs.shape[0]
    x = torch.empty((max(n, 1), FEAT), dtype=torch.bfloat16, device=qcodes.device)
    p = params.c()
    _p._check("pastis_pair_features_qt", _lib().pastis_pair_features_qt(
        ctx.h, _p._ptr(qcodes), _p._ptr(qoffsets), _p._ptr(tcodes), _p._ptr(toffsets), _p._ptr(pairs), n,
        ctypes.byref(p), _p._ptr(x)))
    return x[:n]


def forward(ctx, net: MLP, x: torch.Tensor) -> torch.Tensor:
    n = x.shape[0]
    z = torch.empty(max(n, 1), dtype=torch.float32, device=x.device)
    m = net.c()
    _p._check("pastis_mlp_forward", _lib().pastis_mlp_forward(ctx.h, ctypes.byref(m), _p._ptr(x), n, _p._ptr(z)))
    return z[:n]


def train_step(ctx, net: MLP, x: torch.Tensor, y: torch.Tensor, lr: float, pos_weight: float,
               loss: torch.Tensor = None):
    m = net.c()
    _p._check("pastis_mlp_train_step", _lib().pastis_mlp_train_step(
        ctx.h, ctypes.byref(m), _p._ptr(x), _p._ptr(y), x.shape[0], lr, pos_weight, _p._ptr(loss)))
    net.step = int(m.step)


def select(ctx, pairs: torch.Tensor, logits: torch.Tensor, threshold: float) -> torch.Tensor:
    n = pairs.shape[0]
    nout = ctypes.c_int64()
    out = torch.empty((max(n, 1), _p.REC_BYTES), dtype=torch.uint8, device=pairs.device)
    _p._check("pastis_prefilter_select", _lib().pastis_prefilter_select(
        ctx.h, _p._ptr(pairs), _p._ptr(logits), n, float(threshold), _p._ptr(out), max(n, 1), ctypes.byref(nout)))
    return out[:nout.value]


def labels_from(alns: torch.Tensor) -> torch.Tensor:
    """1.0 where the exact alignment passes the filter (byte 17 of pastis_aln)."""
    return alns[:, 17].float()


def train(ctx, net: MLP, x: torch.Tensor, y: torch.Tensor, epochs=3, batch=65536, lr=2e-3, pos_weight=None,
          seed=0):
    """Minibatch Adam over (x, y); returns the per-epoch mean losses."""
    n = x.shape[0]
    pos = float(y.sum().item())
    if pos_weight is None:
        pos_weight = max(1.0, math.sqrt((n - pos) / max(pos, 1.0)))
    g = torch.Generator(device=x.device).manual_seed(seed)
    loss = torch.zeros(1, device=x.device)
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(n, device=x.device, generator=g)
        tot = 0.0
        steps = 0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            train_step(ctx, net, x[idx].contiguous(), y[idx].contiguous(), lr, pos_weight, loss)
            tot += float(loss.item())
            steps += 1
        hist.append(tot / max(steps, 1))
    return hist


def threshold_for_recall(logits: torch.Tensor, y: torch.Tensor, recall: float) -> float:
    """The largest threshold that keeps at least `recall` of the positives."""
    pz = logits[y > 0.5].float()
    if pz.numel() == 0:
        return float("-inf")
    k = int(math.floor((1.0 - recall) * pz.numel()))
    s = torch.sort(pz).values
    return float(s[k].item()) if k < s.numel() else float(s[-1].item())
