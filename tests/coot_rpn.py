"""Test adapter: build a library expression from an RPN program string (the
oracle's program format), so one string drives both the GPU path and the
oracle.  Uses only the library's public Python API."""
import paper_2508_11385_gb300 as coot

_RED = {"accu", "sum:0", "sum:1", "sum", "mean", "mean:0", "mean:1", "dot", "norm", "norm:fro", "var", "var:0",
        "var:1", "stddev", "stddev:1"}
_STATS = {"min": "min", "max": "max", "index_min": "index_min", "index_max": "index_max", "prod": "prod"}


def is_reduction(tok: str) -> bool:
    if tok in _RED or tok in ("cumsum", "cumsum:0", "cumsum:1"):
        return True
    head, _, rest = tok.partition(":")
    if head in _STATS:
        return rest in ("", "0", "1")
    if head in ("vardim", "stddevdim"):
        parts = rest.split(":")
        return len(parts) == 2 and parts[0] in ("0", "1") and parts[1] in ("0", "1")
    return False


def _reduction(tok, x):
    head, _, rest = tok.partition(":")
    if head == "cumsum":
        return coot.cumsum(x, int(rest) if rest else None)
    if head in _STATS:
        return getattr(coot, _STATS[head])(x, int(rest) if rest else -1)
    if head in ("vardim", "stddevdim"):
        d, n = map(int, rest.split(":"))
        return (coot.var if head == "vardim" else coot.stddev)(x, n, d)
    return {"accu": lambda e: coot.accu(e), "sum": lambda e: coot.sum(e, -1),
            "sum:0": lambda e: coot.sum(e, 0), "sum:1": lambda e: coot.sum(e, 1),
            "mean": lambda e: coot.mean(e, -1), "mean:0": lambda e: coot.mean(e, 0),
            "mean:1": lambda e: coot.mean(e, 1), "norm": lambda e: coot.norm(e),
            "norm:fro": lambda e: coot.norm(e, "fro"), "var": lambda e: coot.var(e, 0),
            "var:0": lambda e: coot.var(e, 0), "var:1": lambda e: coot.var(e, 1),
            "stddev": lambda e: coot.stddev(e, 0), "stddev:1": lambda e: coot.stddev(e, 1)}[tok](x)


def build(program: str, tensors):
    """Returns (expr, reduction or None)."""
    mats = [coot.Mat(t) for t in tensors]
    st = []
    red = None
    for tok in program.split():
        if len(tok) == 1 and "A" <= tok <= "H":
            st.append(mats[ord(tok) - ord("A")])
        elif tok.startswith("#"):
            st.append(float(tok[1:]))
        elif tok in ("+", "-", "%", "/", "*"):
            y = st.pop()
            x = st.pop()
            st.append({"+": lambda a, b: a + b, "-": lambda a, b: a - b, "%": lambda a, b: a % b,
                       "/": lambda a, b: a / b, "*": lambda a, b: a * b}[tok](x, y))
        elif tok == "neg":
            st.append(-st.pop())
        elif tok in ("exp", "log", "abs", "square", "sqrt", "trans"):
            st.append(getattr(coot, tok)(st.pop()))
        elif tok.startswith("each_col:"):
            st.append(coot.broadcast_col(st.pop(), int(tok.split(":")[1])))
        elif tok.startswith("each_row:"):
            st.append(coot.broadcast_row(st.pop(), int(tok.split(":")[1])))
        elif tok == "diag" or tok.startswith("diag:"):
            st.append(st.pop().diag(int(tok.split(":")[1]) if ":" in tok else 0))
        elif tok.startswith("submat:"):
            r0, c0, nr, nc = map(int, tok.split(":")[1:])
            st.append(st.pop().submat(r0, c0, r0 + nr - 1, c0 + nc - 1))
        elif is_reduction(tok):
            if tok == "dot":
                b = st.pop()
                a = st.pop()
                red = coot.dot(a, b)
            else:
                red = _reduction(tok, st.pop())
            st.append(red.expr)
        else:
            raise ValueError(tok)
    assert len(st) == 1
    return st[0], red
