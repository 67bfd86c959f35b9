import numpy as np
def dft_small(v, R, s):
    n=len(v); out=[]
    for k in range(R):
        out.append(sum(v[m]*np.exp(s*2j*np.pi*m*k/R) for m in range(R)))
    return out
def dft3(v,s):
    c=-0.5; sn=0.86602540378443864676
    a,b,d=v; t=b+d; u=a+c*t; w=1j*s*sn*(b-d)
    return [a+t,u+w,u-w]
def dft5(v,s):
    c1=0.30901699437494742410; c2=-0.80901699437494742410; s1=0.95105651629515357212; s2=0.58778525229247312917
    a=v[0]; p1=v[1]+v[4]; m1=v[1]-v[4]; p2=v[2]+v[3]; m2=v[2]-v[3]
    r1=a+c1*p1+c2*p2; r2=a+c2*p1+c1*p2
    q1=1j*s*(s1*m1+s2*m2); q2=1j*s*(s2*m1-s1*m2)
    return [a+p1+p2, r1+q1, r2+q2, r2-q2, r1-q1]
def dft4(v,s):
    t0=v[0]+v[2]; t1=v[0]-v[2]; t2=v[1]+v[3]; t3=1j*s*(v[1]-v[3])
    return [t0+t2, t1+t3, t0-t2, t1-t3]
def plan(n):
    r=[]; m=n
    while m%4==0: r.append(4); m//=4
    while m%2==0: r.append(2); m//=2
    while m%3==0: r.append(3); m//=3
    while m%5==0: r.append(5); m//=5
    assert m==1
    return r
def stockham(x, sign):
    n=len(x); tw=np.exp(-2j*np.pi*np.arange(n)/n)
    src=x.astype(complex).copy(); dst=np.zeros(n,complex); Ns=1
    for R in plan(n):
        nb=n//R; twstep=n//(Ns*R)
        for j in range(nb):
            k=j%Ns
            v=[src[j+m*nb] for m in range(R)]
            if Ns>1:
                for m in range(1,R):
                    w=tw[(m*k*twstep)%n]
                    if sign>0: w=np.conj(w)
                    v[m]*=w
            v = {2:lambda v,s:[v[0]+v[1],v[0]-v[1]],3:dft3,4:dft4,5:dft5}[R](v,sign)
            base=(j//Ns)*Ns*R+k
            for m in range(R): dst[base+m*Ns]=v[m]
        src,dst=dst,src; Ns*=R
    return src
# check small dfts against definition
for R,f in [(3,dft3),(4,dft4),(5,dft5)]:
    v=list(np.random.randn(R)+1j*np.random.randn(R))
    for s in (-1,1):
        assert np.allclose(f(v,s), dft_small(v,R,s)), (R,s)
for n in [2,3,4,5,6,8,12,90,576,300,1280,160,45,2048]:
    x=np.random.randn(n)+1j*np.random.randn(n)
    assert np.allclose(stockham(x,-1), np.fft.fft(x)), n
    assert np.allclose(stockham(x,1), np.fft.ifft(x)*n), n
print("stockham ok")
# packing check
N=576
a=np.random.randn(N); b=np.random.randn(N)
Z=np.fft.fft(a+1j*b)
Zc=np.conj(Z[(-np.arange(N))%N])
A=(Z+Zc)/2; B=(Z-Zc)/(2j)
assert np.allclose(A[:N//2+1], np.fft.rfft(a)) and np.allclose(B[:N//2+1], np.fft.rfft(b))
# inverse packing
Ah=np.fft.rfft(a); Bh=np.fft.rfft(b)
k=np.arange(N); Af=np.where(k<=N//2, Ah[np.minimum(k,N//2)], np.conj(Ah[(N-k)%N if True else 0][...] if False else np.conj(Ah[np.minimum((N-k)%N,N//2)])))
