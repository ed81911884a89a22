/* One node's shell sums, fields and collision with push streaming, in the
 * arithmetic of the FP32 tiled kernel: deviation fields, (+e, -e) pair weights
 * with the exact divided difference of the closure, accumulators in table
 * order, second-order forcing with the A-term.  Included by column.c once per
 * precision variant: TW is the type of the pair weights, accumulators and
 * forces, TC the type of the collision, FETCH the neighbour loader of type TW.
 * Q+ - Q- takes the kernel's form, odd under swapping the pair's ends bit for
 * bit, or (QD_ASYM) the earlier G+ (dn+ - dn-) + (G+ - G-) n-.  CORR adds the
 * kernel's in-plane momentum correction of the FP32 collision in slits (the
 * double sum here stands for its double-word sum). */
        TW noff=(TW)NOFF, hoff=(TW)HOFF, hr = hoff + (TW)hb[z], s0 = (TW)1 - hr - hoff;
        TW me_dn=(TW)nudn[z], vx=(TW)nuv[0][z], vy=(TW)nuv[1][z], vz=(TW)nuv[2][z];
        TW Vx=0,Vy=0,Vz=0,Wx=0,Wy=0,Wz=0,Sxx=0,Syy=0,Szz=0,Sxy=0,Sxz=0,Syz=0,t=0;
        for(int m=0;m<NP;m++){
            TW dnp,hp,vp[3],dnm,hm,vm[3]; FETCH(z+PE[m][2],&dnp,&hp,vp); FETCH(z-PE[m][2],&dnm,&hm,vm);
            TW gnoff=(TW)noff, gs0=(TW)s0, ghp=(TW)hp, ghm=(TW)hm, gdnp=(TW)dnp, gdnm=(TW)dnm;
            TW np=gnoff+gdnp, nm=gnoff+gdnm, sp=gs0-ghp, sm=gs0-ghm, spm=sp*sm, sp2=sp*sp, sm2=sm*sm;
            TW rp=(TW)1/(sp2*sp), rm=(TW)1/(sm2*sm);
            TW gp=fma(sp,rp,rp), gm=fma(sm,rm,rm);
            TW gd=(ghp-ghm)*((sp2+sm2)+fma(spm,sp+sm,spm))*(rp*rm);
            TW qp=gp*np, qm=gm*nm, qd=QD_ASYM ? fma(gp,gdnp-gdnm,gd*nm) : (TW)0.5*fma(gp+gm,gdnp-gdnm,gd*(np+nm));
            TW kx=(TW)PK[m][0], ky=(TW)PK[m][1], kz=(TW)PK[m][2];
            TW px=qp*(TW)vp[0],py=qp*(TW)vp[1],pz=qp*(TW)vp[2];
            TW dx=fma(-qm,(TW)vm[0],px),dy=fma(-qm,(TW)vm[1],py),dz=fma(-qm,(TW)vm[2],pz);
            TW ex=fma(qm,(TW)vm[0],px),ey=fma(qm,(TW)vm[1],py),ez=fma(qm,(TW)vm[2],pz);
            TW tq=qp+qm; t+=tq;
            TW sx=fma(-tq,(TW)vx,ex),sy=fma(-tq,(TW)vy,ey),sz=fma(-tq,(TW)vz,ez);
            Vx=fma((TW)kx,(TW)qd,Vx);Vy=fma((TW)ky,(TW)qd,Vy);Vz=fma((TW)kz,(TW)qd,Vz);
            TW ks=fma(kx,sx,fma(ky,sy,kz*sz));
            Wx=fma((TW)kx,(TW)ks,Wx);Wy=fma((TW)ky,(TW)ks,Wy);Wz=fma((TW)kz,(TW)ks,Wz);
            Sxx=fma((TW)kx,(TW)dx,Sxx);Syy=fma((TW)ky,(TW)dy,Syy);Szz=fma((TW)kz,(TW)dz,Szz);
            Sxy=fma((TW)ky,(TW)dx,fma((TW)kx,(TW)dy,Sxy));Sxz=fma((TW)kz,(TW)dx,fma((TW)kx,(TW)dz,Sxz));Syz=fma((TW)kz,(TW)dy,fma((TW)ky,(TW)dz,Syz));
        }
        TW n = (TW)noff + (TW)me_dn, wh=(TW)0.5*(TW)WSH, mf=-(TW)(1.0/3)*(TW)SIG2*wh*n, vi=(TW)BETA*wh*n, ovx=(TW)vx, ovy=(TW)vy, ovz=(TW)vz;
        TW Cx=mf*(TW)Vx+vi*(TW)Wx, Cy=mf*(TW)Vy+vi*(TW)Wy, Cz=mf*(TW)Vz+vi*(TW)Wz;
        TW pa=-((TW)(1.0/3)/(TW)5)*(TW)SIG2*n*wh;
        TW Axx=(TW)2*pa*((TW)Sxx-(TW)Vx*ovx),Ayy=(TW)2*pa*((TW)Syy-(TW)Vy*ovy),Azz=(TW)2*pa*((TW)Szz-(TW)Vz*ovz);
        TW Axy=pa*((TW)Sxy-((TW)Vy*ovx+(TW)Vx*ovy)),Axz=pa*((TW)Sxz-((TW)Vz*ovx+(TW)Vx*ovz)),Ayz=pa*((TW)Syz-((TW)Vz*ovy+(TW)Vy*ovz));
        TW tsum=(TW)t*wh;
        // collision
        TC cnoff=(TC)NOFF, dsc=nscale[z], sc=cnoff+dsc, d[Q], dn=0, j[3]={0,0,0};
        for(int q=0;q<Q;q++){d[q]=(TC)f[cur][q][z];dn+=d[q];for(int a=0;a<3;a++)if(C[q][a])j[a]+=(TC)C[q][a]*d[q];}
        TC nn=sc+dn, inv=(TC)1/nn;
        TC F[3]={nn*(TC)GX+(TC)Cx, (TC)Cy, (TC)Cz};
        XF_INNER += (double)Cx; XF_DRIVE += (double)(nn*(TC)GX);
        TC u[3]; for(int a=0;a<3;a++) u[a]=(j[a]+(TC)0.5*F[a])*inv;
        TC om=(TC)(1.0/TAU), tr3=((TC)Axx+(TC)Ayy+(TC)Azz)*(TC)(1.0/3);
        TC Bxx=(TC)Axx-tr3,Byy=(TC)Ayy-tr3,Bzz=(TC)Azz-tr3, kA=(TC)2*(TC)4.5;
        TC uu=u[0]*u[0]+u[1]*u[1]+u[2]*u[2], uF=u[0]*F[0]+u[1]*F[1]+u[2]*F[2], src=(TC)1-(TC)0.5*om;
        TC dn_self=(TC)me_dn;
        /* post-collision values; with CORR in the corrected kernel's form,
         * post = d + change, and the changes' in-plane momentum summed */
        TC post_all[Q]; double Mx=0, My=0;
        for(int q=0;q<Q;q++){
            TC wq=(TC)W[q], cu=(TC)C[q][0]*u[0]+(TC)C[q][1]*u[1]+(TC)C[q][2]*u[2], cF=(TC)C[q][0]*F[0]+(TC)C[q][1]*F[1]+(TC)C[q][2]*F[2];
            TC feq=wq*(dn+nn*((TC)3*cu+(TC)4.5*cu*cu-(TC)1.5*uu)), phi=wq*((TC)3*(cF-uF)+(TC)9*cu*cF);
            TC cAc=(TC)(C[q][0]*C[q][0])*Bxx+(TC)(C[q][1]*C[q][1])*Byy+(TC)(C[q][2]*C[q][2])*Bzz+(TC)(2*C[q][0]*C[q][1])*(TC)Axy+(TC)(2*C[q][0]*C[q][2])*(TC)Axz+(TC)(2*C[q][1]*C[q][2])*(TC)Ayz;
            if (CORR) {
                TC dl=src*(phi+kA*wq*cAc)-om*(d[q]-feq);
                post_all[q]=d[q]+dl;
                Mx+=(double)C[q][0]*(double)dl; My+=(double)C[q][1]*(double)dl;
            } else {
                post_all[q]=d[q]-om*(d[q]-feq)+src*(phi+kA*wq*cAc);
            }
        }
        if (CORR) {
            /* the kernel's in-plane momentum correction: the changes' x and y
             * momentum (F exactly) summed without rounding error, and
             * 3 w_q c_q . (F - sum) added back */
            TC ex=(TC)3*(TC)((double)F[0]-Mx), ey=(TC)3*(TC)((double)F[1]-My);
            for(int q=0;q<Q;q++) if(C[q][0]||C[q][1])
                post_all[q]=(TC)fma((double)W[q], (double)((TC)C[q][0]*ex+(TC)C[q][1]*ey), (double)post_all[q]);
        }
        for(int q=0;q<Q;q++){
            TC wq=(TC)W[q], post=post_all[q];
            int zt=z+C[q][2], dst=zt, qq=q; TC dnt;
            if(zt==0||zt==NZ-1){dst=z;qq=OPP[q];dnt=dn_self;} else dnt = (q==0)?dn_self:(TC)nudn[zt];
            f[nxt][qq][dst] = (STORE)(post + wq*(dsc-dnt));
        }
        new_nscale[z] = (double)dn_self;
        cprev[0][z] = (STORE)Cx; cprev[1][z] = (STORE)Cy; cprev[2][z] = (STORE)Cz; tprev[z] = (STORE)tsum;
